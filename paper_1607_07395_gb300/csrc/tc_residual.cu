// Step a9 on tensor cores -- the exact relative Frobenius error
// |A - U diag(S) V^T|_F / |A|_F of Section 5, fused and tiled.
//
// A_hat = (U diag(S)) V^T is a contraction with K = k, so it runs on tcgen05:
// the operands (U diag(S) and V, rounded to BF16 or kept as TF32, K padded
// with zeros to a multiple of the 128-byte swizzle width) are staged by TMA,
// a 128 x 256 (BF16) or 128 x 128 (TF32) tile of A_hat accumulates in TMEM,
// and the epilogue warps read it back with tcgen05.ld while they stream the
// same tile of A from HBM once, summing (a - a_hat)^2 and a^2 (FP32 within a
// tile, FP64 across tiles: FP64 runs at 1/64 of the FP32 rate here). A_hat
// is never written. A CTA keeps one column block of V resident and walks the
// row tiles of that block, so V is read from L2 once per CTA and U diag(S)
// once per column block. Per-CTA sums are added in a fixed order.
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
__global__ void residual_prep_kernel(const float* __restrict__ U, const double* __restrict__ S,
                                     const float* __restrict__ V, long long m, long long n, int k, int Kp,
                                     void* __restrict__ USp, void* __restrict__ Vp) {
  const long long total = (m + n) * Kp;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long row = e / Kp;
    const int r = (int)(e - row * Kp);
    float v = 0.f;
    if (r < k) v = row < m ? (float)((double)U[row * k + r] * S[r]) : V[(row - m) * k + r];
    if constexpr (kTF32) {
      (row < m ? (float*)USp : (float*)Vp)[(row < m ? row : row - m) * Kp + r] = v;
    } else {
      (row < m ? (__nv_bfloat16*)USp : (__nv_bfloat16*)Vp)[(row < m ? row : row - m) * Kp + r] = __float2bfloat16_rn(v);
    }
  }
}

template <bool kTF32>
__global__ void __launch_bounds__(tc::kThreads, 1)
    tc_residual_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                       const float* __restrict__ Amat, long long lda, int m, int n, int nch, int units,
                       double* __restrict__ part, int* err) {
  using Cfg = ResCfg<kTF32>;
  constexpr int BN = Cfg::BN;
  extern __shared__ uint8_t smem_raw[];
  __shared__ tc::Barriers bars;
  __shared__ double red[2][tc::kEpiWarps];
  uint8_t *Bres, *Aring;
  tc::setup<BN>(smem_raw, nch, Bres, Aring, &bars);
  const int MT = (m + tc::kBM - 1) / tc::kBM;
  const int u0 = (int)((long long)units * blockIdx.x / gridDim.x);
  const int u1 = (int)((long long)units * (blockIdx.x + 1) / gridDim.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == 0) {
    if (lane == 0) {
      tc::prefetch_tmap(&tmA);
      tc::prefetch_tmap(&tmB);
      tc::producer_loop<BN>(&tmA, &tmB, Bres, Aring, &bars, u0, u1, MT, nch, Cfg::KC);
    }
  } else if (warp == 1) {
    if (lane == 0) tc::mma_loop<kTF32, BN>(Bres, Aring, &bars, u0, u1, MT, nch);
  } else if (warp >= tc::kEpiWarp0) {
    const int e = warp - tc::kEpiWarp0;
    const int sub = warp & 3;             // TMEM lane quarter
    const int half = e >> 2;              // column half
    const int row = sub * 32 + lane;      // tile row
    const bool vec = ((lda & 3) == 0) && (((uintptr_t)Amat & 15) == 0);
    double num = 0.0, den = 0.0;
    int ab = 0;
    uint32_t accph[2] = {0, 0};
    for (int u = u0; u < u1; ++u) {
      int cb, rt;
      tc::unit_of(u, MT, cb, rt);
      if (!tc::mbar_wait(&bars.accfull[ab], accph[ab], &bars.abort)) break;
      accph[ab] ^= 1;
      tc::fence_after_sync();
      const long long gi = (long long)rt * tc::kBM + row;
      const bool row_ok = gi < m;
      const float* arow = Amat + (row_ok ? gi : 0) * lda;
      float tn = 0.f, td = 0.f;  // FP32 within a tile (<= 128 terms), FP64 across tiles
      constexpr int NJ = BN / 2 / 32;
      float a[2][32];
      auto load_chunk = [&](int j, float (&dst)[32]) {
        const long long gc0 = (long long)cb * BN + half * (BN / 2) + j * 32;
        if (row_ok && vec && gc0 + 32 <= n) {
          const float4* p4 = (const float4*)(arow + gc0);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const float4 t = __ldg(p4 + q);
            dst[4 * q] = t.x;
            dst[4 * q + 1] = t.y;
            dst[4 * q + 2] = t.z;
            dst[4 * q + 3] = t.w;
          }
        } else {
#pragma unroll
          for (int q = 0; q < 32; ++q) dst[q] = (row_ok && gc0 + q < n) ? __ldg(arow + gc0 + q) : 0.f;
        }
      };
      load_chunk(0, a[0]);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        if (j + 1 < NJ) load_chunk(j + 1, a[(j + 1) & 1]);  // next chunk's loads in flight
        const int c0 = half * (BN / 2) + j * 32;
        const long long gc0 = (long long)cb * BN + c0;
        float v[32];
        tc::tmem_ld32(bars.tmem_base + (uint32_t)(ab * BN + c0) + ((uint32_t)(sub * 32) << 16), v);
        if (row_ok) {
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            if (gc0 + q < n) {
              const float x = a[j & 1][q];
              const float dl = x - v[q];
              tn = fmaf(dl, dl, tn);
              td = fmaf(x, x, td);
            }
          }
        }
      }
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
              residual_prep_kernel<kTF32><<<std::max(1, std::min(ceil_div((m + n) * Kp, 256), sm_count() * 8)), 256,
                                            0, stream>>>(U, S, V, m, n, k, Kp, USp, Vp));
  if (cudaMemsetAsync(err, 0, sizeof(int), stream) != cudaSuccess) return check_cuda("tc residual err clear");
  const size_t smem = tc::smem_bytes(nch, Cfg::BN);
  cudaFuncSetAttribute(tc_residual_kernel<kTF32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  CABS_LAUNCH(stream, "tc_residual_kernel",
              tc_residual_kernel<kTF32><<<grid, tc::kThreads, smem, stream>>>(
                  tmA, tmB, (const float*)src.A, src.lda, (int)m, (int)n, nch, units, part, err));
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
