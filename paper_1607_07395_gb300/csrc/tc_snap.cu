// Step a6 on tensor cores -- candidate rows for the snap of Section 3.2 in
// the BF16 and TF32 modes.
//
// Every centre z_j needs its nearest rows of P (or Q). Ranking the rows of
// one centre by |x|^2 - 2 x . z gives the same order as |x - z|^2 (|z|^2 is a
// per-centre constant), so the contraction x . z for all centres and all rows
// runs on tcgen05: the centres (k2 <= 256, one or two 128-row tiles) stream
// through the TMA ring as the A operand and a block of 256 rows stays
// resident as the B operand; the 128 x 256 FP32 accumulator of a unit
// (centre tile, row block) lives in TMEM, double-buffered. In the epilogue a
// thread owns one centre (its TMEM lane) and keeps the kTopTc smallest
// approximate values over its half of the block in registers; the two halves
// merge through shared memory and the block's list is stored.
//
// The approximate order only chooses candidates. tc_snap_merge_kernel takes
// each centre's kPool best approximate candidates over all blocks, recomputes
// their distances by direct differences with exactly the arithmetic of the
// CUDA-core candidate kernel (one thread per row, FP32 fused multiply-adds in
// dimension order) and keeps the 8 nearest in (distance, row) order. Whenever
// those 8 are among the kPool, the lists, and so the greedy walk, equal the
// CUDA-core ones bit for bit.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "profile.cuh"
#include "tc_assign.cuh"
#include "tc_gemm.cuh"
#include "tc_snap.cuh"

namespace cabs {
namespace {

constexpr int kBN = 256;     // rows of P per resident block
constexpr int kTopTc = 8;    // approximate candidates per (centre, block)
constexpr int kMergeList = 16;  // per-thread list of the merge (>= its share of a centre's candidates)
constexpr int kPool = 32;    // approximate candidates per centre re-ranked exactly
constexpr int kTopOut = 8;   // exact candidates per centre handed to the greedy pass

template <bool kTF32>
struct SnapCfg {
  static constexpr int KC = kTF32 ? 32 : 64;
  static constexpr int ES = kTF32 ? 4 : 2;
};

// Keeps (d, r) sorted ascending by (value, row); static indices only.
template <int N>
__device__ __forceinline__ void topn_insert(float (&d)[N], int (&r)[N], float v, int row) {
  if (!(v < d[N - 1] || (v == d[N - 1] && row < r[N - 1]))) return;
  d[N - 1] = v;
  r[N - 1] = row;
#pragma unroll
  for (int i = N - 1; i > 0; --i) {
    if (d[i] < d[i - 1] || (d[i] == d[i - 1] && r[i] < r[i - 1])) {
      const float td = d[i];
      d[i] = d[i - 1];
      d[i - 1] = td;
      const int tr = r[i];
      r[i] = r[i - 1];
      r[i - 1] = tr;
    }
  }
}

__global__ void row_norms_kernel(const float* __restrict__ X, long long M, int d, float* __restrict__ xn) {
  const int lane = threadIdx.x & 31;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long l = warp; l < M; l += nwarps) {
    float s = 0.f;
    for (int q = lane; q < d; q += 32) s = fmaf(X[l * d + q], X[l * d + q], s);
    s = warp_sum(s);
    if (lane == 0) xn[l] = s;
  }
}

template <bool kTF32>
__global__ void __launch_bounds__(tc::kThreads, 1)
    tc_snap_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const float* __restrict__ xn, int M, int k2, int nch, int MT, int units,
                   float* __restrict__ cand_d, int* __restrict__ cand_r, int* err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ tc::Barriers bars;
  __shared__ float xd[4][kTopTc][32];
  __shared__ int xr[4][kTopTc][32];
  uint8_t *Bres, *Aring;
  tc::setup<kBN>(smem_raw, nch, Bres, Aring, &bars);
  const int u0 = (int)((long long)units * blockIdx.x / gridDim.x);
  const int u1 = (int)((long long)units * (blockIdx.x + 1) / gridDim.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      tc::prefetch_tmap(&tmA);
      tc::prefetch_tmap(&tmB);
      tc::producer_loop<kBN>(&tmA, &tmB, Bres, Aring, &bars, u0, u1, MT, nch, SnapCfg<kTF32>::KC);
    }
  } else if (warp == 1) {
    if (lane == 0) tc::mma_loop<kTF32, kBN>(Bres, Aring, &bars, u0, u1, MT, nch);
  } else if (warp >= tc::kEpiWarp0) {
    const int e = warp - tc::kEpiWarp0;
    const int sub = warp & 3, half = e >> 2;
    const int row = sub * 32 + lane;
    int ab = 0;
    uint32_t accph[2] = {0, 0};
    for (int u = u0; u < u1; ++u) {
      int cb, rt;
      tc::unit_of(u, MT, cb, rt);
      // every epilogue warp must leave together: they share named barrier 1
      const int fail = tc::mbar_wait(&bars.accfull[ab], accph[ab], &bars.abort) ? 0 : 1;
      int anyfail;
      asm volatile(
          "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 q, %1, 0;\n\t"
          "bar.red.or.pred p, 1, %2, q;\n\tselp.s32 %0, 1, 0, p;\n\t}"
          : "=r"(anyfail)
          : "r"(fail), "n"(tc::kEpiWarps * 32));
      if (anyfail) break;
      accph[ab] ^= 1;
      tc::fence_after_sync();
      float bd[kTopTc];
      int br[kTopTc];
#pragma unroll
      for (int t = 0; t < kTopTc; ++t) {
        bd[t] = __int_as_float(0x7f800000);
        br[t] = 0x7fffffff;
      }
#pragma unroll 1
      for (int c = 0; c < kBN / 2 / 32; ++c) {
        const int col0 = half * (kBN / 2) + c * 32;
        const long long p0 = (long long)cb * kBN + col0;
        if (p0 >= M) break;  // warp-uniform
        float v[32];
        tc::tmem_ld32(bars.tmem_base + (uint32_t)(ab * kBN + col0) + ((uint32_t)(sub * 32) << 16), v);
        const float xl = p0 + lane < M ? __ldg(xn + p0 + lane) : 0.f;
        // one pass marks the values below this centre's current 8th best
        // (a superset: the bound only falls as values enter), then only those
        // are inserted, rows rising, each checked against the bound of the
        // moment -- the same list as inserting every value in turn
        float dv[32];
        unsigned cand = 0u;
        const float bound = bd[kTopTc - 1];
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const float xq = __shfl_sync(0xffffffffu, xl, q);
          dv[q] = p0 + q < M ? fmaf(-2.f, v[q], xq) : __int_as_float(0x7f800000);
          cand |= dv[q] < bound ? (1u << q) : 0u;
        }
        while (cand) {
          const int q = __ffs(cand) - 1;
          cand &= cand - 1u;
          topn_insert<kTopTc>(bd, br, dv[q], (int)(p0 + q));
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.accempty[ab]);
      ab ^= 1;
      // merge the two column halves of each centre (warps w and w + 4)
      if (half == 1) {
#pragma unroll
        for (int t = 0; t < kTopTc; ++t) {
          xd[sub][t][lane] = bd[t];
          xr[sub][t][lane] = br[t];
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(tc::kEpiWarps * 32));
      if (half == 0) {
#pragma unroll
        for (int t = 0; t < kTopTc; ++t) topn_insert<kTopTc>(bd, br, xd[sub][t][lane], xr[sub][t][lane]);
        const int j = rt * tc::kBM + row;
        if (j < k2) {
          const size_t o = ((size_t)cb * k2 + j) * kTopTc;
#pragma unroll
          for (int t = 0; t < kTopTc; ++t) {
            cand_d[o + t] = bd[t];
            cand_r[o + t] = br[t];
          }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(tc::kEpiWarps * 32));
    }
  }
  tc::teardown<kBN>(&bars, err);
}

// One CTA (256 threads) per centre j: the kPool smallest approximate values
// over all blocks, then direct FP32 distances for those rows and the kTopOut
// nearest in (distance, row) order.
__global__ void __launch_bounds__(256) tc_snap_merge_kernel(const float* __restrict__ cand_d,
                                                            const int* __restrict__ cand_r, int nblk, int k2,
                                                            const float* __restrict__ X, long long M, int d,
                                                            const float* __restrict__ Z, float* __restrict__ top_d,
                                                            int* __restrict__ top_r) {
  __shared__ float wd[8];
  __shared__ int wr[8], wt[8];
  __shared__ int win_t;
  __shared__ int pool_r[kPool];
  __shared__ float pool_x[kPool];
  const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wi = tid >> 5;
  float bd[kMergeList];
  int br[kMergeList];
#pragma unroll
  for (int t = 0; t < kMergeList; ++t) {
    bd[t] = __int_as_float(0x7f800000);
    br[t] = 0x7fffffff;
  }
  const long long total = (long long)nblk * kTopTc;
  for (long long e = tid; e < total; e += blockDim.x) {
    const long long b = e / kTopTc, t = e - b * kTopTc;
    const size_t o = ((size_t)b * k2 + j) * kTopTc + t;
    const int r = cand_r[o];
    if (r >= 0 && r < M) topn_insert<kMergeList>(bd, br, cand_d[o], r);
  }
  // kPool rounds of a block-wide arg-min over the threads' list heads
  for (int round = 0; round < kPool; ++round) {
    float v = bd[0];
    int r = br[0];
    int who = tid;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, v, off);
      const int orr = __shfl_xor_sync(0xffffffffu, r, off);
      const int ow = __shfl_xor_sync(0xffffffffu, who, off);
      if (ov < v || (ov == v && orr < r)) {
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
      float bv = wd[0];
      int brr = wr[0], bw = wt[0];
      for (int i = 1; i < 8; ++i)
        if (wd[i] < bv || (wd[i] == bv && wr[i] < brr)) {
          bv = wd[i];
          brr = wr[i];
          bw = wt[i];
        }
      pool_r[round] = brr;
      win_t = bw;
    }
    __syncthreads();
    if (tid == win_t) {  // pop the head
#pragma unroll
      for (int t = 0; t < kMergeList - 1; ++t) {
        bd[t] = bd[t + 1];
        br[t] = br[t + 1];
      }
      bd[kMergeList - 1] = __int_as_float(0x7f800000);
      br[kMergeList - 1] = 0x7fffffff;
    }
    __syncthreads();
  }
  // distances of the pool, one thread per row, as the CUDA-core kernel sums them
  const float* z = Z + (size_t)j * d;
  if (tid < kPool) {
    const int r = pool_r[tid];
    float s = 0.f;
    const bool valid = r >= 0 && r < M;
    if (valid)
      for (int q = 0; q < d; ++q) {
        const float df = X[(long long)r * d + q] - z[q];
        s = fmaf(df, df, s);
      }
    pool_x[tid] = valid ? s : __int_as_float(0x7f800000);
  }
  __syncthreads();
  if (wi == 0) {
    const float v = pool_x[lane];
    const int r = pool_r[lane];
    int rank = 0;
    for (int t = 0; t < kPool; ++t) {
      const float ov = pool_x[t];
      const int orr = pool_r[t];
      rank += (ov < v || (ov == v && orr < r) || (ov == v && orr == r && t < lane)) ? 1 : 0;
    }
    if (rank < kTopOut) {
      const bool valid = r >= 0 && r < M;
      top_d[(size_t)j * kTopOut + rank] = valid ? v : __int_as_float(0x7f800000);
      top_r[(size_t)j * kTopOut + rank] = valid ? r : 0x7fffffff;
    }
  }
}

struct TcSnapWs {
  void *Pp, *Zp;
  float* xn;
  float* cand_d;
  int* cand_r;
  int* err;
};

TcSnapWs carve_tc_snap(Carve& cv, int64_t M, int d, int k2) {
  const int Kp = tc_kp_of(d, true);  // sized for the wider (TF32) operands
  const int nblk = ceil_div(M, kBN);
  TcSnapWs w;
  w.Pp = cv.take<char>((size_t)M * Kp * 4);
  w.Zp = cv.take<char>((size_t)kBN * Kp * 4);
  w.xn = cv.take<float>(M);
  w.cand_d = cv.take<float>((size_t)nblk * k2 * kTopTc);
  w.cand_r = cv.take<int>((size_t)nblk * k2 * kTopTc);
  w.err = cv.take<int>(1);
  return w;
}

template <bool kTF32>
cabs_status tc_snap_typed(const float* X, int64_t M, int d, const float* Z, int k2, float* top_d, int* top_r,
                          void* ws, size_t ws_bytes, cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  TcSnapWs w = carve_tc_snap(cv, M, d, k2);
  if (!cv.fits()) {
    set_error("tensor-core snap workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  const int Kp = tc_kp_of(d, kTF32);
  const int nch = Kp / SnapCfg<kTF32>::KC;
  const int sms = sm_count();
  CABS_TRY(tc_to_operand(X, M, d, Kp, kTF32, w.Pp, "tc_snap_points_prep", stream));
  CABS_TRY(tc_to_operand(Z, k2, d, Kp, kTF32, w.Zp, "tc_snap_centres_prep", stream));
  CABS_LAUNCH(stream, "row_norms_kernel",
              row_norms_kernel<<<std::max(1, std::min(ceil_div(M, 8), sms * 16)), 256, 0, stream>>>(X, M, d, w.xn));
  if (cudaMemsetAsync(w.err, 0, sizeof(int), stream) != cudaSuccess) return check_cuda("tc_snap err clear");
  CUtensorMap tmA, tmB;
  const int dt = kTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CABS_TRY(make_tmap_2d(&tmA, w.Zp, dt, k2, Kp, (uint64_t)Kp * SnapCfg<kTF32>::ES, SnapCfg<kTF32>::KC, tc::kBM));
  CABS_TRY(make_tmap_2d(&tmB, w.Pp, dt, M, Kp, (uint64_t)Kp * SnapCfg<kTF32>::ES, SnapCfg<kTF32>::KC, kBN));
  const int nblk = ceil_div(M, kBN);
  const int MT = ceil_div(k2, tc::kBM);
  const int units = nblk * MT;
  const int grid = std::max(1, std::min(units, sms));
  const size_t smem = tc::smem_bytes(nch, kBN);
  cudaFuncSetAttribute(tc_snap_kernel<kTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  CABS_LAUNCH(stream, "tc_snap_kernel",
              tc_snap_kernel<kTF32><<<grid, tc::kThreads, smem, stream>>>(tmA, tmB, w.xn, (int)M, k2, nch, MT,
                                                                        units, w.cand_d, w.cand_r, w.err));
  CABS_LAUNCH(stream, "tc_snap_merge_kernel",
              tc_snap_merge_kernel<<<k2, 256, 0, stream>>>(w.cand_d, w.cand_r, nblk, k2, X, M, d, Z, top_d, top_r));
  return CABS_OK;
}

}  // namespace

bool tc_snap_supported(int64_t M, int d, int k2, bool tf32) {
  const int Kp = tc_kp_of(d, tf32);
  const int nch = Kp / (tf32 ? 32 : 64);
  // the merge's per-thread lists hold every candidate a thread scans: at most
  // ceil(nblk kTopTc / 256) <= kMergeList, i.e. M <= 131072 rows
  const long long nblk = (M + kBN - 1) / kBN;
  return M >= 1 && (nblk * kTopTc + 255) / 256 <= kMergeList && k2 >= 1 && k2 <= kBN &&
         (size_t)nch * kBN * 128 <= 128 * 1024;
}

size_t tc_snap_ws_bytes(int64_t M, int d, int k2) {
  Carve cv;
  carve_tc_snap(cv, M, d, k2);
  return cv.used;
}

cabs_status tc_snap_candidates(const float* X, int64_t M, int d, const float* Z, int k2, bool tf32, float* top_d,
                               int* top_r, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (tf32) return tc_snap_typed<true>(X, M, d, Z, k2, top_d, top_r, ws, ws_bytes, stream);
  return tc_snap_typed<false>(X, M, d, Z, k2, top_d, top_r, ws, ws_bytes, stream);
}

}  // namespace cabs
