// Step a6 -- every k-means centre is replaced by its closest in-sample point
// (Section 3.2, last paragraph), giving the follow-up indices of Algorithm 2,
// step 3.
//
// Centres are taken in index order and each takes the nearest row not taken
// before (ties to the lower row index), so the k2 follow-up rows are
// distinct. Distances are direct differences sum_q (x_q - z_q)^2 in the
// working precision, summed in dimension order (the same arithmetic in every
// kernel below, so equal inputs give equal distances).
//
//  1. snap_cand_kernel: a CTA covers 64 rows x all centres (register tiles of
//     8 x 8 per thread) and keeps, per centre, its 8 nearest rows of the tile.
//  2. snap_merge_kernel: one CTA per centre merges the tile lists into the
//     centre's global 8 nearest rows, ordered by (distance, row).
//  3. snap_greedy_kernel: one CTA walks the centres in order; warp 0 picks the
//     first candidate not taken (a bitmap of taken rows in shared memory);
//     only if all 8 are taken does the whole CTA scan every row for that
//     centre. The picks are then sorted ascending.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace cabs {
namespace {

constexpr int kTop = 8;
constexpr int kSM = 64, kSK = 16, kSN = 256;
constexpr int kGreedyThreads = 1024;
constexpr size_t kBitmapSmemLimit = 160 * 1024;

template <typename T>
__device__ __forceinline__ void top_insert(T (&d)[kTop], int (&r)[kTop], T v, int row) {
  if (!lex_less(v, row, d[kTop - 1], r[kTop - 1])) return;
  int i = kTop - 1;
  while (i > 0 && lex_less(v, row, d[i - 1], r[i - 1])) {
    d[i] = d[i - 1];
    r[i] = r[i - 1];
    --i;
  }
  d[i] = v;
  r[i] = row;
}

template <typename T>
__global__ void __launch_bounds__(256) snap_cand_kernel(const T* __restrict__ X, long long M, int d,
                                                        const T* __restrict__ Z, int k2, T* __restrict__ cand_d,
                                                        int* __restrict__ cand_r) {
  extern __shared__ __align__(16) unsigned char snap_smem[];
  T* xs = (T*)snap_smem;                 // [kSK][kSM + 1]
  T* zs = xs + kSK * (kSM + 1);          // [kSK][kSN + 1]
  T* dist = (T*)snap_smem;               // reused after the contraction: [kSM][kSN + 1]
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  const long long m0 = (long long)blockIdx.x * kSM;
  T acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[i][c] = T(0);
  for (int q0 = 0; q0 < d; q0 += kSK) {
    for (int e = tid; e < kSM * kSK; e += 256) {
      const int p = e / kSK, qq = e - p * kSK;
      const long long l = m0 + p;
      const int q = q0 + qq;
      xs[qq * (kSM + 1) + p] = (l < M && q < d) ? X[l * d + q] : T(0);
    }
    for (int e = tid; e < kSN * kSK; e += 256) {
      const int j = e / kSK, qq = e - j * kSK;
      const int q = q0 + qq;
      zs[qq * (kSN + 1) + j] = (j < k2 && q < d) ? Z[(size_t)j * d + q] : T(0);
    }
    __syncthreads();
    const int kq = min(kSK, d - q0);
    const int nc = (k2 + 31) >> 5;  // centre columns in use (the rest are padding)
    for (int kk = 0; kk < kq; ++kk) {
      T a[8], b[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = xs[kk * (kSM + 1) + ty * 8 + i];
#pragma unroll
      for (int c = 0; c < 8; ++c) b[c] = zs[kk * (kSN + 1) + tx + 32 * c];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        if (c < nc) {
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const T t = a[i] - b[c];
            acc[i][c] = fma(t, t, acc[i][c]);
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int c = 0; c < 8; ++c) dist[(ty * 8 + i) * (kSN + 1) + tx + 32 * c] = acc[i][c];
  __syncthreads();
  const int j = tid;
  if (j < k2) {
    T bd[kTop];
    int br[kTop];
#pragma unroll
    for (int t = 0; t < kTop; ++t) {
      bd[t] = pos_inf<T>();
      br[t] = 0x7fffffff;
    }
    for (int p = 0; p < kSM; ++p) {
      const long long l = m0 + p;
      if (l < M) top_insert(bd, br, dist[p * (kSN + 1) + j], (int)l);
    }
    const size_t o = ((size_t)blockIdx.x * k2 + j) * kTop;
#pragma unroll
    for (int t = 0; t < kTop; ++t) {
      cand_d[o + t] = bd[t];
      cand_r[o + t] = br[t];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256) snap_merge_kernel(const T* __restrict__ cand_d, const int* __restrict__ cand_r,
                                                         int nblk, int k2, T* __restrict__ top_d,
                                                         int* __restrict__ top_r) {
  __shared__ T wd[8];
  __shared__ int wr[8], wt[8];
  __shared__ int win_t;
  const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
  T bd[kTop];
  int br[kTop];
#pragma unroll
  for (int t = 0; t < kTop; ++t) {
    bd[t] = pos_inf<T>();
    br[t] = 0x7fffffff;
  }
  const long long total = (long long)nblk * kTop;
  for (long long e = tid; e < total; e += blockDim.x) {
    const long long b = e / kTop, t = e - b * kTop;
    const size_t o = ((size_t)b * k2 + j) * kTop + t;
    top_insert(bd, br, cand_d[o], cand_r[o]);
  }
  int head = 0;
  for (int round = 0; round < kTop; ++round) {
    T v = head < kTop ? bd[head] : pos_inf<T>();
    int r = head < kTop ? br[head] : 0x7fffffff;
    int who = tid;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const T ov = __shfl_xor_sync(0xffffffffu, v, off);
      const int orr = __shfl_xor_sync(0xffffffffu, r, off);
      const int ow = __shfl_xor_sync(0xffffffffu, who, off);
      if (lex_less(ov, orr, v, r)) {
        v = ov;
        r = orr;
        who = ow;
      }
    }
    if (lane == 0) {
      wd[wi] = v;
      wr[wi] = r;
      wt[wi] = who;
    }
    __syncthreads();
    if (tid == 0) {
      T bv = wd[0];
      int brr = wr[0], bw = wt[0];
      for (int i = 1; i < 8; ++i)
        if (lex_less(wd[i], wr[i], bv, brr)) {
          bv = wd[i];
          brr = wr[i];
          bw = wt[i];
        }
      top_d[(size_t)j * kTop + round] = bv;
      top_r[(size_t)j * kTop + round] = brr;
      win_t = bw;
    }
    __syncthreads();
    if (tid == win_t) ++head;
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(kGreedyThreads) snap_greedy_kernel(const T* __restrict__ X, long long M, int d,
                                                                      const T* __restrict__ Z, int k2,
                                                                      const int* __restrict__ top_r, int use_smem,
                                                                      unsigned* bitmap_g, int* __restrict__ order,
                                                                      int* __restrict__ sorted, int* fallbacks) {
  extern __shared__ __align__(16) unsigned bm_smem[];
  __shared__ int picks[CABS_MAX_K];
  __shared__ int fb_j;
  __shared__ T wd[32];
  __shared__ int wr[32];
  unsigned* taken = use_smem ? bm_smem : bitmap_g;
  const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5, nw = blockDim.x >> 5;
  const long long words = (M + 31) / 32;
  for (long long e = tid; e < words; e += blockDim.x) taken[e] = 0u;
  __syncthreads();
  int j = 0;
  while (j < k2) {
    if (wi == 0) {
      // warp 0 resolves centres from its candidate lists until one needs a full scan
      int jj = j;
      for (; jj < k2; ++jj) {
        const int r = lane < kTop ? top_r[(size_t)jj * kTop + lane] : 0x7fffffff;
        const bool ok = lane < kTop && r >= 0 && r < M && !((taken[r >> 5] >> (r & 31)) & 1u);
        const unsigned good = __ballot_sync(0xffffffffu, ok);
        if (!good) break;
        const int first = __ffs(good) - 1;
        const int pick = __shfl_sync(0xffffffffu, r, first);
        if (lane == 0) {
          taken[pick >> 5] |= 1u << (pick & 31);
          picks[jj] = pick;
        }
        __syncwarp();
      }
      if (lane == 0) fb_j = jj;
    }
    __syncthreads();
    j = fb_j;
    if (j >= k2) break;
    // full scan for centre j over the rows not taken yet
    T best = pos_inf<T>();
    int brow = 0x7fffffff;
    const T* z = Z + (size_t)j * d;
    for (long long l = tid; l < M; l += blockDim.x) {
      if ((taken[l >> 5] >> (l & 31)) & 1u) continue;
      T s = T(0);
      for (int q = 0; q < d; ++q) {
        const T t = X[l * d + q] - z[q];
        s = fma(t, t, s);
      }
      if (lex_less(s, (int)l, best, brow)) {
        best = s;
        brow = (int)l;
      }
    }
    warp_argmin(best, brow);
    if (lane == 0) {
      wd[wi] = best;
      wr[wi] = brow;
    }
    __syncthreads();
    if (tid == 0) {
      T bv = wd[0];
      int bi = wr[0];
      for (int i = 1; i < nw; ++i)
        if (lex_less(wd[i], wr[i], bv, bi)) {
          bv = wd[i];
          bi = wr[i];
        }
      if (bi >= 0 && bi < M) taken[bi >> 5] |= 1u << (bi & 31);
      picks[j] = bi;
      if (fallbacks) atomicAdd(fallbacks, 1);
    }
    __syncthreads();
    ++j;
  }
  __syncthreads();
  for (int i = tid; i < k2; i += blockDim.x) order[i] = picks[i];
  // rank sort of the distinct picks
  for (int i = tid; i < k2; i += blockDim.x) {
    const int v = picks[i];
    int r = 0;
    for (int t = 0; t < k2; ++t) r += picks[t] < v;
    sorted[r] = v;
  }
}

struct SnapWs {
  void* cand_d;
  int* cand_r;
  void* top_d;
  int* top_r;
  unsigned* bitmap;
};

SnapWs carve_snap(Carve& cv, int64_t M, int k2, size_t eb) {
  SnapWs w;
  const int nblk = ceil_div(M, kSM);
  w.cand_d = cv.take<char>((size_t)nblk * k2 * kTop * eb);
  w.cand_r = cv.take<int>((size_t)nblk * k2 * kTop);
  w.top_d = cv.take<char>((size_t)k2 * kTop * eb);
  w.top_r = cv.take<int>((size_t)k2 * kTop);
  w.bitmap = cv.take<unsigned>((size_t)(M + 31) / 32);
  return w;
}

template <typename T>
cabs_status snap_typed(const T* X, int64_t M, int d, const T* Z, int k2, int* order, int* sorted, void* ws,
                       size_t ws_bytes, int* fallbacks, cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  SnapWs w = carve_snap(cv, M, k2, sizeof(T));
  if (!cv.fits()) {
    set_error("snap workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  const int nblk = ceil_div(M, kSM);
  const size_t stage = (size_t)(kSK * (kSM + 1) + kSK * (kSN + 1)) * sizeof(T);
  const size_t dtile = (size_t)kSM * (kSN + 1) * sizeof(T);
  const size_t smem = std::max(stage, dtile);
  cudaFuncSetAttribute(snap_cand_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  CABS_LAUNCH(stream, "snap_cand_kernel", snap_cand_kernel<T><<<nblk, 256, smem, stream>>>(X, M, d, Z, k2, (T*)w.cand_d, w.cand_r));
  CABS_LAUNCH(stream, "snap_merge_kernel", snap_merge_kernel<T><<<k2, 256, 0, stream>>>((const T*)w.cand_d, w.cand_r, nblk, k2, (T*)w.top_d, w.top_r));
  const size_t bm_bytes = (size_t)((M + 31) / 32) * 4;
  const int use_smem = bm_bytes <= kBitmapSmemLimit;
  const size_t gsm = use_smem ? bm_bytes : 0;
  if (gsm > 48 * 1024)
    cudaFuncSetAttribute(snap_greedy_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  CABS_LAUNCH(stream, "snap_greedy_kernel", snap_greedy_kernel<T><<<1, kGreedyThreads, gsm, stream>>>(X, M, d, Z, k2, w.top_r, use_smem, w.bitmap, order,
                                                            sorted, fallbacks));
  return CABS_OK;
}

}  // namespace

size_t snap_ws_bytes(int64_t M, int d, int k2, int prec) {
  Carve cv;
  carve_snap(cv, M, k2, elem_bytes(prec));
  return cv.used;
}

cabs_status launch_snap(const void* X, int64_t M, int d, const void* Z, int k2, int prec, int* order, int* sorted,
                        void* ws, size_t ws_bytes, int* fallbacks, cudaStream_t stream) {
  if (prec == CABS_PREC_FP64)
    return snap_typed<double>((const double*)X, M, d, (const double*)Z, k2, order, sorted, ws, ws_bytes, fallbacks,
                              stream);
  return snap_typed<float>((const float*)X, M, d, (const float*)Z, k2, order, sorted, ws, ws_bytes, fallbacks,
                           stream);
}

}  // namespace cabs
