// Step a9 on tensor cores -- the exact relative Frobenius error
// |A - U diag(S) V^T|_F / |A|_F of Section 5, fused and tiled.
//
// A_hat = (U diag(S)) V^T is a contraction with K = k, so it runs on tcgen05:
// the operands (U diag(S) and V, rounded to BF16 or kept as TF32, K padded
// with zeros to a multiple of the 128-byte swizzle width) are staged by TMA,
// a 128 x 256 (BF16) or 128 x 128 (TF32) tile of A_hat accumulates in TMEM
// (two accumulators, so one tile's epilogue overlaps the next tile's MMAs).
// A itself is streamed from HBM once, by TMA as well: a fourth role (warp 3)
// loads each tile of A as 128-row x 32-column chunks (128-byte swizzle) into
// a ring, so the epilogue warps read their row of a chunk from shared memory
// without bank conflicts, while the copies keep HBM busy. The epilogue sums
// (a - a_hat)^2 and a^2 in FP32 within a tile and in FP64 across tiles (FP64
// runs at 1/64 of the FP32 rate here). A_hat is never written. A CTA keeps
// one column block of V resident and walks the row tiles of that block, so V
// is read from L2 once per CTA and U diag(S) once per column block. Per-CTA
// sums are added in a fixed order.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "tc_gemm.cuh"

namespace cabs {
namespace {

template <bool kTF32>
struct ResCfg {
  static constexpr int BN = kTF32 ? 128 : 256;
  static constexpr int KC = kTF32 ? 32 : 64;  // elements per 128-byte K chunk
  static constexpr int ES = kTF32 ? 4 : 2;
};

// US_p[i][r] = U[i][r] S[r], V_p[j][r] = V[j][r] for r < k; zero for k <= r < Kp.
template <bool kTF32>
__global__ void __launch_bounds__(256) residual_prep_kernel(const float* __restrict__ U, const double* __restrict__ S,
                                                            const float* __restrict__ V, long long m, long long n,
                                                            int k, int Kp, void* __restrict__ USp,
                                                            void* __restrict__ Vp) {
  // one warp per row, lanes along the row (coalesced); U diag(S) in FP32
  // before the rounding to the operand type, whose unit roundoff dominates
  __shared__ float s32[CABS_MAX_K];
  for (int r = threadIdx.x; r < k; r += blockDim.x) s32[r] = (float)S[r];
  __syncthreads();
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  for (long long row = (long long)blockIdx.x * wpb + (threadIdx.x >> 5); row < m + n;
       row += (long long)gridDim.x * wpb) {
    const bool top = row < m;
    const long long rr = top ? row : row - m;
    const float* src = (top ? U : V) + rr * k;
    for (int r = lane; r < Kp; r += 32) {
      const float v = r < k ? (top ? src[r] * s32[r] : src[r]) : 0.f;
      if constexpr (kTF32) {
        ((float*)(top ? USp : Vp))[rr * Kp + r] = v;
      } else {
        ((__nv_bfloat16*)(top ? USp : Vp))[rr * Kp + r] = __float2bfloat16_rn(v);
      }
    }
  }
}

constexpr int kUSt = 2;                          // ring stages of U diag(S) row tiles
// Ring stages of A chunks. The producer alternates the two column halves and
// each unit has an even number of chunks, so with an even stage count every
// slot always serves the same half: a group of epilogue warps then waits on a
// slot's next phase only after it consumed the previous one. (With an odd
// count the halves would alternate on a slot, and a group could wait for
// phase n + 1 while the slot is still in phase n, which a parity wait cannot
// tell apart from phase n - 1 completing.)
constexpr int kMSt = 4;
static_assert(kMSt % 2 == 0, "each A slot must serve one column half");
constexpr uint32_t kMChunkBytes = tc::kBM * 128; // one A chunk: 128 rows x 32 FP32 columns

// Waits for a phase regardless of the abort flag (bounded): used to let the
// copies a role has issued land before the CTA exits.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < tc::kWaitLimit; ++i)
    if (tc::mbar_try_wait(bar, parity)) return;
}

template <bool kTF32>
__global__ void __launch_bounds__(tc::kThreads, 1)
    tc_residual_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const __grid_constant__ CUtensorMap tmM, int m, int nch, int units,
                       double* __restrict__ part, int* err) {
  using Cfg = ResCfg<kTF32>;
  constexpr int BN = Cfg::BN;
  constexpr int NC = BN / 32;  // A chunks per unit
  extern __shared__ uint8_t smem_raw[];
  __shared__ tc::Barriers bars;
  __shared__ uint64_t mfull[kMSt], mempty[kMSt];
  __shared__ double red[2][tc::kEpiWarps];
  if (threadIdx.x == 0) {
    for (int i = 0; i < kMSt; ++i) {
      tc::mbar_init(&mfull[i], 1);
      tc::mbar_init(&mempty[i], 4);  // the 4 warps of one column half read a slot
    }
  }
  uint8_t *Bres, *Aring;
  tc::setup<BN>(smem_raw, nch, Bres, Aring, &bars);
  uint8_t* Mring = Aring + (size_t)kUSt * tc::kBM * 128;
  const int MT = (m + tc::kBM - 1) / tc::kBM;
  const int u0 = (int)((long long)units * blockIdx.x / gridDim.x);
  const int u1 = (int)((long long)units * (blockIdx.x + 1) / gridDim.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      tc::prefetch_tmap(&tmA);
      tc::prefetch_tmap(&tmB);
      tc::producer_loop<BN, kUSt>(&tmA, &tmB, Bres, Aring, &bars, u0, u1, MT, nch, Cfg::KC);
    }
  } else if (warp == 1) {
    if (lane == 0) tc::mma_loop<kTF32, BN, kUSt>(Bres, Aring, &bars, u0, u1, MT, nch);
  } else if (warp == 3) {
    // A producer: the unit's A tile as NC chunks of 32 columns, interleaving
    // the two column halves so both groups of epilogue warps progress
    if (lane == 0) {
      tc::prefetch_tmap(&tmM);
      long long issued = 0;
      bool ok = true;
      for (int u = u0; u < u1 && ok; ++u) {
        int cb, rt;
        tc::unit_of(u, MT, cb, rt);
        for (int t = 0; t < NC; ++t) {
          const int c = (t & 1) * (NC / 2) + (t >> 1);
          const int s = (int)(issued % kMSt);
          const uint32_t ph = (uint32_t)((issued / kMSt) & 1);
          if (!tc::mbar_wait(&mempty[s], ph ^ 1, &bars.abort)) {
            ok = false;
            break;
          }
          tc::mbar_expect_tx(&mfull[s], kMChunkBytes);
          tc::tma_load_2d(Mring + (size_t)s * kMChunkBytes, &tmM, &mfull[s], cb * BN + c * 32, rt * tc::kBM);
          ++issued;
        }
      }
      if (!ok)  // let the copies in flight land before the CTA exits
        for (long long j = issued > kMSt ? issued - kMSt : 0; j < issued; ++j)
          mbar_drain(&mfull[j % kMSt], (uint32_t)((j / kMSt) & 1));
    }
  } else if (warp >= tc::kEpiWarp0) {
    const int e = warp - tc::kEpiWarp0;
    const int sub = warp & 3;             // TMEM lane quarter
    const int half = e >> 2;              // column half
    const int row = sub * 32 + lane;      // tile row
    double num = 0.0, den = 0.0;
    int ab = 0;
    uint32_t accph[2] = {0, 0};
    long long ubase = 0;  // A chunks of the units before this one
    bool ok = true;
    for (int u = u0; u < u1 && ok; ++u) {
      if (!tc::mbar_wait(&bars.accfull[ab], accph[ab], &bars.abort)) break;
      accph[ab] ^= 1;
      tc::fence_after_sync();
      // Out-of-range rows and columns are zero in A (TMA fill) and in the
      // contraction (zero operand rows), so they add nothing.
      float tn = 0.f, td = 0.f;  // FP32 within a tile (<= 128 terms), FP64 across tiles
#pragma unroll 1
      for (int j = 0; j < NC / 2; ++j) {
        const int c = half * (NC / 2) + j;
        const long long i = ubase + 2 * j + half;
        const int s = (int)(i % kMSt);
        if (!tc::mbar_wait(&mfull[s], (uint32_t)((i / kMSt) & 1), &bars.abort)) {
          ok = false;
          break;
        }
        // 128-byte swizzle: 16-byte group q of row r sits at q ^ (r % 8)
        const uint8_t* rp = Mring + (size_t)s * kMChunkBytes + (size_t)row * 128;
        float a[32];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 t = *(const float4*)(rp + ((q ^ (row & 7)) << 4));
          a[4 * q] = t.x;
          a[4 * q + 1] = t.y;
          a[4 * q + 2] = t.z;
          a[4 * q + 3] = t.w;
        }
        float v[32];
        tc::tmem_ld32(bars.tmem_base + (uint32_t)(ab * BN + c * 32) + ((uint32_t)(sub * 32) << 16), v);
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const float dl = a[q] - v[q];
          tn = fmaf(dl, dl, tn);
          td = fmaf(a[q], a[q], td);
        }
        // release the slot only once every lane has consumed its values, so no
        // shared-memory read of this chunk can still be pending when the
        // producer's next copy lands in it
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&mempty[s]);
      }
      ubase += NC;
      num += (double)tn;
      den += (double)td;
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.accempty[ab]);
      ab ^= 1;
    }
    num = warp_sum(num);
    den = warp_sum(den);
    if (lane == 0) {
      red[0][e] = num;
      red[1][e] = den;
    }
  }
  tc::teardown<BN>(&bars, err);
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int i = 0; i < tc::kEpiWarps; ++i) {
      s0 += red[0][i];
      s1 += red[1][i];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

__global__ void tc_pair_reduce_kernel(const double* __restrict__ part, int nb, const int* __restrict__ err,
                                      double* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += part[2 * i];
    b += part[2 * i + 1];
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int off = 128; off > 0; off >>= 1) {
    if ((int)threadIdx.x < off) {
      s0[threadIdx.x] += s0[threadIdx.x + off];
      s1[threadIdx.x] += s1[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    // a kernel that gave up a wait reports NaN rather than a partial sum
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    out[0] = *err ? nan : s0[0];
    out[1] = *err ? nan : s1[0];
  }
}

template <bool kTF32>
cabs_status tc_residual_typed(const cabs_source& src, int64_t m, int64_t n, int k, const float* U, const double* S,
                              const float* V, void* ws, size_t ws_bytes, double* out2, cudaStream_t stream) {
  using Cfg = ResCfg<kTF32>;
  const int Kp = (k + Cfg::KC - 1) / Cfg::KC * Cfg::KC;
  const int nch = Kp / Cfg::KC;
  const int MT = ceil_div(m, tc::kBM), NBt = ceil_div(n, Cfg::BN);
  const int units = MT * NBt;
  const int grid = std::max(1, std::min(units, sm_count()));
  Carve cv(ws, ws_bytes);
  void* USp = cv.take<char>((size_t)m * Kp * Cfg::ES);
  void* Vp = cv.take<char>((size_t)n * Kp * Cfg::ES);
  double* part = cv.take<double>((size_t)2 * grid);
  int* err = cv.take<int>(1);
  if (!cv.fits()) {
    set_error("tensor-core residual workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  CUtensorMap tmA, tmB;
  const int dt = kTF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CABS_TRY(make_tmap_2d(&tmA, USp, dt, m, Kp, (uint64_t)Kp * Cfg::ES, Cfg::KC, tc::kBM));
  CABS_TRY(make_tmap_2d(&tmB, Vp, dt, n, Kp, (uint64_t)Kp * Cfg::ES, Cfg::KC, Cfg::BN));
  CABS_LAUNCH(stream, "tc_residual_prep",
              residual_prep_kernel<kTF32><<<std::max(1, std::min(ceil_div(m + n, 8), sm_count() * 8)), 256, 0,
                                            stream>>>(U, S, V, m, n, k, Kp, USp, Vp));
  if (cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess) return check_cuda("tc residual err clear");
  CUtensorMap tmM;
  CABS_TRY(make_tmap_2d(&tmM, src.A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, m, n, (uint64_t)src.lda * 4, 32, tc::kBM));
  const size_t smem = tc::smem_bytes<kUSt>(nch, Cfg::BN) + (size_t)kMSt * kMChunkBytes;
  cudaFuncSetAttribute(tc_residual_kernel<kTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  CABS_LAUNCH(stream, "tc_residual_kernel",
              tc_residual_kernel<kTF32><<<grid, tc::kThreads, smem, stream>>>(tmA, tmB, tmM, (int)m, nch, units,
                                                                            part, err));
  CABS_LAUNCH(stream, "tc_pair_reduce_kernel", tc_pair_reduce_kernel<<<1, 256, 0, stream>>>(part, grid, err, out2));
  return CABS_OK;
}

}  // namespace

size_t tc_residual_ws_bytes(int64_t m, int64_t n, int k, bool tf32) {
  const int KC = tf32 ? 32 : 64, ES = tf32 ? 4 : 2;
  const int Kp = (k + KC - 1) / KC * KC;
  Carve cv;
  cv.take<char>((size_t)m * Kp * ES);
  cv.take<char>((size_t)n * Kp * ES);
  cv.take<double>((size_t)2 * 1024);
  cv.take<int>(1);
  return cv.used;
}

cabs_status launch_tc_residual(const cabs_source& src, int64_t m, int64_t n, int k, bool tf32, const float* U,
                               const double* S, const float* V, void* ws, size_t ws_bytes, double* out2,
                               cudaStream_t stream) {
  if (tf32) return tc_residual_typed<true>(src, m, n, k, U, S, V, ws, ws_bytes, out2, stream);
  return tc_residual_typed<false>(src, m, n, k, U, S, V, ws, ws_bytes, out2, stream);
}

}  // namespace cabs
