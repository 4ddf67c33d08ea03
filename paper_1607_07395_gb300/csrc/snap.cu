// Step a6 -- every k-means centre is replaced by its closest in-sample point
// (Section 3.2, last paragraph), giving the follow-up indices of Algorithm 2,
// step 3.
//
// Centres are taken in index order and each takes the nearest row not taken
// before, so the k2 follow-up rows are distinct. Ties go to the lower row
// index, a tie meaning a squared distance within tie_rtol (d* + |z|^2) of the
// nearest untaken row's d*: the centre of a two-row cluster is the midpoint
// of the rows, exactly equidistant from both, and which rounded distance is
// smaller would otherwise depend on the order of the sum. Distances are
// direct differences sum_q (x_q - z_q)^2 in the working precision.
//
//  1. snap_cand_kernel: a CTA covers 64 rows x all centres (register tiles of
//     8 x 8 per thread) and keeps, per centre, its 8 nearest rows of the tile.
//  2. snap_merge_kernel: one CTA per centre merges the tile lists into the
//     centre's global 8 nearest rows, ordered by (distance, row).
//     In the BF16 and TF32 modes steps 1-2 run on tensor cores instead
//     (tc_snap.cu): the 32 best rows per centre by |x|^2 - 2 x.z, then the
//     same direct FP32 distances as step 1 decide the 8 candidates.
//  3. snap_greedy_kernel (cooperative): CTA 0's warp 0 walks the centres in
//     order and picks the lowest untaken candidate inside the tie window of
//     the first untaken one (taken rows in shared memory); only if all 8 are taken,
//     or the window reaches the 8th, do all CTAs scan every row for that
//     centre. The picks are then sorted ascending.
#include "common.cuh"
#include "grid_sync.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "tc_snap.cuh"

namespace cabs {
namespace {

constexpr int kTop = 8;
// Tie window of the snap (relative to d* + |z|^2): the centre of a two-row
// cluster is equidistant from both rows, and the rounded distances differ by
// at most about 2 u (d* + |z|^2) plus the summation error (u the unit
// roundoff, up to d u for d dimensions). FP64: 1e-12 (35 times 256 u);
// FP32 (every reduced-precision mode decides by FP32 distances): 2^-16.
constexpr double kSnapTieRtolF64 = 1e-12;
constexpr float kSnapTieRtolF32 = 1.52587890625e-5f;
constexpr int kSM = 64, kSK = 16, kSN = 256;
constexpr int kGreedyThreads = 512;

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

// Cooperative greedy pass. CTA 0's warp 0 walks the centres in order. For
// centre j with candidate list (d_0, r_0) <= ... <= (d_7, r_7), let d* be the
// distance of the first candidate not taken yet; the centre takes the lowest
// row among the untaken candidates with d <= d* + tie_rtol (d* + |z_j|^2)
// (rows that tie with the nearest at the working precision's resolution; the
// centre of a two-row cluster is exactly equidistant from both rows). The
// list decides alone when every row outside it is farther than that window,
// i.e. when d_7 lies beyond it. Otherwise -- all 8 taken, or the window
// reaching d_7 -- every CTA scans its slice of rows for centre j (one warp per
// row, lanes over dimensions) in two passes: the nearest untaken row (d*),
// then the lowest untaken row inside the window; CTA 0 reduces the per-CTA
// results in a fixed order and the walk continues.
// Open-addressing set of taken rows (at most CABS_MAX_K of them) in shared
// memory; -1 marks a free slot.
constexpr int kTakenSlots = 4 * CABS_MAX_K;

__device__ __forceinline__ unsigned taken_slot(int r) { return ((unsigned)r * 2654435761u) >> 22; }

__device__ __forceinline__ bool taken_has(const int* set, int r) {
  unsigned s = taken_slot(r);
  for (int probe = 0; probe < kTakenSlots; ++probe, s = (s + 1) & (kTakenSlots - 1)) {
    const int v = set[s];
    if (v == r) return true;
    if (v < 0) return false;
  }
  return false;
}

__device__ __forceinline__ void taken_add(int* set, int r) {
  unsigned s = taken_slot(r);
  for (int probe = 0; probe < kTakenSlots; ++probe, s = (s + 1) & (kTakenSlots - 1)) {
    if (set[s] == r) return;
    if (set[s] < 0) {
      set[s] = r;
      return;
    }
  }
}

// rows per warp and step of a full scan: with the dimension loop unrolled,
// 4 rows keep 32 loads per lane in flight within the kernel's register
// budget (two 512-thread CTAs per SM)
template <typename T>
__host__ __device__ constexpr int scan_rows() { return 4; }
// Rows whose taken set fits in shared memory as a bitmap (16 KB, 131072
// rows): larger inputs keep the open-addressing set of the rows taken so far.
constexpr long long kMaxBitWords = 4096;

// Pass 1 of a full scan: the (distance, row) minimum over rows [lo, hi) not
// in the taken bitmap, for centre z; each computed distance is also stored
// in dist[l] for pass 2.
template <typename T>
__device__ void scan_slice(const T* __restrict__ X, int d, const T* __restrict__ z, long long lo, long long hi,
                           const unsigned* taken, T* __restrict__ dist, T& best, int& brow) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  constexpr int kScanRows_T = scan_rows<T>();
  best = pos_inf<T>();
  brow = 0x7fffffff;
  for (long long l0 = lo + (long long)wi * kScanRows_T; l0 < hi; l0 += (long long)nw * kScanRows_T) {
    bool skip[kScanRows_T];
    T s4[kScanRows_T];
#pragma unroll
    for (int u = 0; u < kScanRows_T; ++u) {
      const long long l = l0 + u;
      skip[u] = l >= hi || ((((volatile const unsigned*)taken)[l >> 5] >> (l & 31)) & 1u);
      s4[u] = T(0);
    }
    // unrolled so that the rows' loads (d <= 256: 8 per row and lane) are in
    // flight together; each lane still sums its dimensions in order
#pragma unroll 8
    for (int q = lane; q < d; q += 32) {
      const T zq = z[q];
#pragma unroll
      for (int u = 0; u < kScanRows_T; ++u) {
        if (!skip[u]) {
          const T t = X[(l0 + u) * d + q] - zq;
          s4[u] = fma(t, t, s4[u]);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kScanRows_T; ++u) {
      const T sv = warp_sum(s4[u]);
      if (skip[u]) continue;
      if (lane == 0) dist[l0 + u] = sv;
      if (lex_less(sv, (int)(l0 + u), best, brow)) {
        best = sv;
        brow = (int)(l0 + u);
      }
    }
  }
}

// Pass 2: the lowest untaken row of [lo, hi) whose pass-1 distance is <= lim
// (one thread per row; +inf, 0x7fffffff if none).
template <typename T>
__device__ void window_slice(long long lo, long long hi, const unsigned* taken, const T* __restrict__ dist, T lim,
                             T& best, int& brow) {
  best = pos_inf<T>();
  brow = 0x7fffffff;
  for (long long l = lo + threadIdx.x; l < hi; l += blockDim.x) {
    if ((((volatile const unsigned*)taken)[l >> 5] >> (l & 31)) & 1u) continue;
    const T v = ((volatile const T*)dist)[l];
    if (v <= lim) {
      best = v;
      brow = (int)l;
      break;  // rows rise with l: the first hit is this thread's lowest
    }
  }
  // lowest row over the warp
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const int orow = __shfl_xor_sync(0xffffffffu, brow, off);
    const T ov = __shfl_xor_sync(0xffffffffu, best, off);
    if (orow < brow) {
      brow = orow;
      best = ov;
    }
  }
}

// Per-CTA result of scan_slice -> cta_best[b], cta_row[b] (pass 1: the lexicographic
// minimum over the warps; pass 2: the lowest row).
template <typename T>
__device__ void cta_reduce(T best, int brow, bool window, T* wd, int* wr, T* cta_best, int* cta_row) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    wd[wi] = best;
    wr[wi] = brow;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    T bv = wd[0];
    int bi = wr[0];
    for (int i = 1; i < nw; ++i)
      if (window ? wr[i] < bi : lex_less(wd[i], wr[i], bv, bi)) {
        bv = wd[i];
        bi = wr[i];
      }
    cta_best[blockIdx.x] = bv;
    cta_row[blockIdx.x] = bi;
  }
}

template <typename T>
__global__ void __launch_bounds__(kGreedyThreads, 2) snap_greedy_kernel(
    const T* __restrict__ X, long long M, int d, const T* __restrict__ Z, int k2, const int* __restrict__ top_r,
    const T* __restrict__ top_d, T tie_rtol, unsigned* taken, int* picks, int* next_fb, T* cta_best, int* cta_row,
    T* fb_lim, T* dist, GridBarrier* bar, int* __restrict__ order, int* __restrict__ sorted, int* fallbacks,
    int* status) {
  __shared__ T wd[kGreedyThreads / 32];
  __shared__ int wr[kGreedyThreads / 32];
  // CTA 0's walk reads the candidate lists, their distances, the centres'
  // squared norms and the rows taken so far from shared memory: the lists
  // are staged once, the taken rows are a bitmap (inputs up to
  // 32 kMaxBitWords rows) or, beyond that, an open-addressing set of
  // kTakenSlots slots (at most k2 rows are ever taken). The global bitmap is
  // written too, for the CTAs' scans when a centre's list does not decide.
  // shared memory: s_topd[k2 kTop], s_zz[k2] (T), s_top[k2 kTop], s_taken (int),
  // then (M <= 32 kMaxBitWords) the taken rows as a bitmap s_bits; static
  // shared memory (at most 46 KB in FP64), so the cooperative launch passes
  // no dynamic size
  __shared__ __align__(16) T s_topd[CABS_MAX_K * kTop];
  __shared__ T s_zz[CABS_MAX_K];
  __shared__ int s_top[CABS_MAX_K * kTop];
  __shared__ int s_taken[kTakenSlots];
  __shared__ unsigned s_bits[kMaxBitWords];
  const int tid = threadIdx.x, lane = tid & 31, wi = tid >> 5, nw = blockDim.x >> 5;
  const unsigned G = gridDim.x;
  const long long words = (M + 31) / 32;
  const bool use_bits = words <= kMaxBitWords;
  auto has = [&](int r) { return use_bits ? ((s_bits[r >> 5] >> (r & 31)) & 1u) != 0u : taken_has(s_taken, r); };
  auto add = [&](int r) {
    if (use_bits)
      s_bits[r >> 5] |= 1u << (r & 31);
    else
      taken_add(s_taken, r);
  };
  // a barrier that gave up: report it (diagnostics status bit 2) and leave
  auto gave_up = [&]() {
    if (tid == 0 && status) atomicOr(status, 4);
  };
  for (long long e = (long long)blockIdx.x * blockDim.x + tid; e < words; e += (long long)G * blockDim.x)
    taken[e] = 0u;
  if (blockIdx.x == 0) {
    for (int e = tid; e < k2 * kTop; e += blockDim.x) {
      s_top[e] = top_r[e];
      s_topd[e] = top_d[e];
    }
    for (int e = tid; e < kTakenSlots; e += blockDim.x) s_taken[e] = -1;
    if (use_bits)
      for (long long e = tid; e < words; e += blockDim.x) s_bits[e] = 0u;
    for (int j = wi; j < k2; j += nw) {
      T s = T(0);
      for (int q = lane; q < d; q += 32) s = fma(Z[(size_t)j * d + q], Z[(size_t)j * d + q], s);
      s = warp_sum(s);
      if (lane == 0) s_zz[j] = s;
    }
  }
  if (!grid_sync(bar, G)) return gave_up();
  int j = 0;
  while (true) {
    if (blockIdx.x == 0 && wi == 0) {
      int jj = j;
      for (; jj < k2; ++jj) {
        const int r = lane < kTop ? s_top[jj * kTop + lane] : 0x7fffffff;
        const T dv = lane < kTop ? s_topd[jj * kTop + lane] : pos_inf<T>();
        const bool ok = lane < kTop && r >= 0 && r < M && !has(r);
        const unsigned good = __ballot_sync(0xffffffffu, ok);
        if (!good) break;
        const T dstar = __shfl_sync(0xffffffffu, dv, __ffs(good) - 1);
        const T lim = dstar + tie_rtol * (dstar + s_zz[jj]);
        const T dlast = __shfl_sync(0xffffffffu, dv, kTop - 1);
        if (dlast <= lim) break;  // rows outside the list may lie inside the window
        int cand = (ok && dv <= lim) ? r : 0x7fffffff;
#pragma unroll
        for (int off = kTop / 2; off > 0; off >>= 1) cand = min(cand, __shfl_xor_sync(0xffffffffu, cand, off));
        if (lane == 0) {
          add(cand);
          // a reduction, not a read-modify-write: the walk does not wait on it
          // (the scans read the bitmap only after the next grid barrier)
          atomicOr(&taken[cand >> 5], 1u << (cand & 31));
          picks[jj] = cand;
        }
        __syncwarp();
      }
      if (lane == 0) *next_fb = jj;
    }
    if (!grid_sync(bar, G)) return gave_up();
    j = *(volatile int*)next_fb;
    if (j >= k2) break;
    // every CTA, pass 1: nearest untaken row of its slice for centre j
    const long long lo = M * blockIdx.x / G, hi = M * (blockIdx.x + 1) / G;
    const T* z = Z + (size_t)j * d;
    T best;
    int brow;
    scan_slice(X, d, z, lo, hi, taken, dist, best, brow);
    cta_reduce(best, brow, false, wd, wr, cta_best, cta_row);
    if (!grid_sync(bar, G)) return gave_up();
    if (blockIdx.x == 0 && tid == 0) {
      T bv = cta_best[0];
      int bi = cta_row[0];
      for (unsigned b = 1; b < G; ++b)
        if (lex_less(cta_best[b], cta_row[b], bv, bi)) {
          bv = cta_best[b];
          bi = cta_row[b];
        }
      *(volatile T*)fb_lim = bv + tie_rtol * (bv + s_zz[j]);
      __threadfence();
    }
    if (!grid_sync(bar, G)) return gave_up();
    // pass 2: lowest untaken row of the slice inside the window
    window_slice(lo, hi, taken, dist, *(volatile T*)fb_lim, best, brow);
    cta_reduce(best, brow, true, wd, wr, cta_best, cta_row);
    if (!grid_sync(bar, G)) return gave_up();
    if (blockIdx.x == 0 && tid == 0) {
      int bi = cta_row[0];
      for (unsigned b = 1; b < G; ++b) bi = min(bi, cta_row[b]);
      if (bi >= 0 && bi < M) {
        atomicOr(&taken[bi >> 5], 1u << (bi & 31));
        add(bi);
      }
      picks[j] = bi;
      if (fallbacks) atomicAdd(fallbacks, 1);
      __threadfence();
    }
    __syncthreads();  // warp 0 of CTA 0 sees the pick before it resumes
    ++j;  // CTA 0's warp 0 resumes at the next centre; the others wait at the next barrier
  }
  if (blockIdx.x == 0) {
    __syncthreads();
    for (int i = tid; i < k2; i += blockDim.x) order[i] = ((volatile int*)picks)[i];
    for (int i = tid; i < k2; i += blockDim.x) {
      const int v = ((volatile int*)picks)[i];
      int r = 0;
      for (int t = 0; t < k2; ++t) r += ((volatile int*)picks)[t] < v;
      sorted[r] = v;
    }
  }
}

__global__ void snap_state_init_kernel(GridBarrier* bar, int* next_fb, long long limit) {
  bar->count = 0u;
  bar->gen = 0u;
  bar->err = 0;
  bar->limit = limit;
  *next_fb = 0;
}

struct SnapWs {
  void* cand_d;
  int* cand_r;
  void* top_d;
  int* top_r;
  unsigned* bitmap;
  int *picks, *next_fb, *cta_row;
  void *cta_best, *fb_lim, *dist;
  GridBarrier* bar;
  void* tc;  // tensor-core candidate search (BF16 / TF32 modes)
  size_t tc_bytes;
};

SnapWs carve_snap(Carve& cv, int64_t M, int d, int k2, int prec) {
  const size_t eb = elem_bytes(prec);
  SnapWs w;
  const int nblk = ceil_div(M, kSM);
  w.cand_d = cv.take<char>((size_t)nblk * k2 * kTop * eb);
  w.cand_r = cv.take<int>((size_t)nblk * k2 * kTop);
  w.top_d = cv.take<char>((size_t)k2 * kTop * eb);
  w.top_r = cv.take<int>((size_t)k2 * kTop);
  w.bitmap = cv.take<unsigned>((size_t)(M + 31) / 32);
  w.picks = cv.take<int>(CABS_MAX_K);
  w.next_fb = cv.take<int>(1);
  w.cta_row = cv.take<int>(1024);
  w.cta_best = cv.take<char>(1024 * eb);
  w.fb_lim = cv.take<char>(eb);
  w.dist = cv.take<char>((size_t)M * eb);
  w.bar = cv.take<GridBarrier>(1);
  w.tc = nullptr;
  w.tc_bytes = 0;
  if (prec == CABS_PREC_BF16 || prec == CABS_PREC_TF32) {
    w.tc_bytes = tc_snap_ws_bytes(M, d, k2);
    w.tc = cv.take<char>(w.tc_bytes);
  }
  return w;
}

template <typename T>
cabs_status snap_typed(const T* X, int64_t M, int d, const T* Z, int k2, int prec, int* order, int* sorted, void* ws,
                       size_t ws_bytes, int* fallbacks, int* status, cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  SnapWs w = carve_snap(cv, M, d, k2, prec);
  if (!cv.fits()) {
    set_error("snap workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  const bool tf32 = prec == CABS_PREC_TF32;
  if (w.tc && sizeof(T) == 4 && tc_snap_supported(M, d, k2, tf32)) {
    // reduced precision: candidates ranked on tensor cores, then by direct distance
    CABS_TRY(tc_snap_candidates((const float*)X, M, d, (const float*)Z, k2, tf32, (float*)w.top_d, w.top_r, w.tc,
                                w.tc_bytes, stream));
  } else {
    const int nblk = ceil_div(M, kSM);
    const size_t stage = (size_t)(kSK * (kSM + 1) + kSK * (kSN + 1)) * sizeof(T);
    const size_t dtile = (size_t)kSM * (kSN + 1) * sizeof(T);
    const size_t smem = std::max(stage, dtile);
    cudaFuncSetAttribute(snap_cand_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    CABS_LAUNCH(stream, "snap_cand_kernel", snap_cand_kernel<T><<<nblk, 256, smem, stream>>>(X, M, d, Z, k2, (T*)w.cand_d, w.cand_r));
    CABS_LAUNCH(stream, "snap_merge_kernel", snap_merge_kernel<T><<<k2, 256, 0, stream>>>((const T*)w.cand_d, w.cand_r, nblk, k2, (T*)w.top_d, w.top_r));
  }
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, snap_greedy_kernel<T>, kGreedyThreads, 0);
  // a CTA per 512 rows, so that a full scan (a centre whose candidates are
  // all taken) has enough loads in flight
  const int G = std::max(1, std::min({(int)ceil_div(M, 512), coop_grid_cap(sm_count() * std::max(per_sm, 1)), 1024}));
  CABS_LAUNCH(stream, "snap_state_init", snap_state_init_kernel<<<1, 1, 0, stream>>>(w.bar, w.next_fb, wait_limit()));
  const T* Xc = X;
  const T* Zc = Z;
  const int* topr = w.top_r;
  const T* topd = (const T*)w.top_d;
  T tie = sizeof(T) == 8 ? T(kSnapTieRtolF64) : T(kSnapTieRtolF32);
  unsigned* bm = w.bitmap;
  int* picks = w.picks;
  int* nfb = w.next_fb;
  T* cb = (T*)w.cta_best;
  int* cr = w.cta_row;
  T* lim = (T*)w.fb_lim;
  T* dst = (T*)w.dist;
  GridBarrier* bar = w.bar;
  long long Ml = M;
  void* args[] = {&Xc, &Ml, &d, &Zc, &k2, &topr, &topd, &tie, &bm, &picks, &nfb, &cb, &cr, &lim, &dst, &bar, &order,
                  &sorted, &fallbacks, &status};
  CABS_LAUNCH(stream, "snap_greedy_kernel",
              cudaLaunchCooperativeKernel((const void*)snap_greedy_kernel<T>, dim3(G), dim3(kGreedyThreads), args,
                                          0, stream));
  return CABS_OK;
}

}  // namespace

size_t snap_ws_bytes(int64_t M, int d, int k2, int prec) {
  Carve cv;
  carve_snap(cv, M, d, k2, prec);
  return cv.used;
}

cabs_status launch_snap(const void* X, int64_t M, int d, const void* Z, int k2, int prec, int* order, int* sorted,
                        void* ws, size_t ws_bytes, int* fallbacks, int* status, cudaStream_t stream) {
  if (prec == CABS_PREC_FP64)
    return snap_typed<double>((const double*)X, M, d, (const double*)Z, k2, prec, order, sorted, ws, ws_bytes,
                              fallbacks, status, stream);
  return snap_typed<float>((const float*)X, M, d, (const float*)Z, k2, prec, order, sorted, ws, ws_bytes, fallbacks,
                           status, stream);
}

}  // namespace cabs
