// Step a4 on tensor cores -- the extrapolation products a = C V_w and
// b = R^T U_w of the sketching routine (Section 4.1) in the BF16 and TF32
// modes, to FP32-level accuracy.
//
// out[M x N] = X[M x K] B[K x N] with X in FP32 (C or R^T, row-major) and B
// the FP64 k x k factor (N = K = k <= 256). Each operand is split as
// x = hi + lo with hi = x rounded to TF32 (11 significant bits) and lo the
// exact FP32 remainder, and the product is taken as three TF32 products on
// tcgen05, X_hi B_hi + X_hi B_lo + X_lo B_hi (the dropped X_lo B_lo is below
// 2^-22 of |x| |b|), accumulated in FP32 in TMEM: a relative error near
// 2^-21 per term, against 2^-11 for a single TF32 product.
//
// One CTA per SM over 128-row tiles, persistent; per tile the K axis runs in
// chunks of 32 values (one 128-byte swizzled row per operand row). Roles:
//   warps 0-3   producers: coalesced loads of the X chunk (a warp per 32
//               rows, a lane per column), written as hi and lo straight into
//               the stage's 128-byte-swizzled A buffers (any K: no TMA row
//               alignment rule applies); thread 0 also bulk-copies the
//               chunk's B_hi / B_lo images into the stage;
//   warp 4      one thread issues the 12 MMAs of a chunk (M = 128, N = Np,
//               K = 8 each) into one of two TMEM accumulators;
//   warp 5      allocates / frees TMEM;
//   warps 8-11  epilogue: lane = TMEM lane = tile row; stores the row and the
//               FP64 sum of squares of each column over the tile's 128 rows
//               (part[tile * N + col], the same 128-row blocks as the
//               CUDA-core kernel), in a fixed order.
// The B images (B_hi, B_lo of both products, each chunk in its swizzled
// shared-memory layout) are written once per core by a small prep kernel.
// Every wait is bounded (tc::mbar_wait); on a timeout all roles leave, the
// CTA sets bit 2 of *err and frees its TMEM.
#include "kernels.cuh"
#include "profile.cuh"
#include "tc_common.cuh"

namespace cabs {
namespace {

constexpr int kXBM = 128;       // rows per tile = TMEM lanes
constexpr int kXStages = 2;
constexpr int kXThreads = 384;
constexpr int kXProd = 128;     // producer threads (warps 0-3)
constexpr int kXMmaWarp = 4;
constexpr int kXTmemWarp = 5;
constexpr int kXEpi0 = 8;       // epilogue warps 8-11 (TMEM lane quarters 0-3)

struct alignas(8) XBars {
  uint64_t full[kXStages];      // 128 producer arrivals + the B bytes
  uint64_t empty[kXStages];     // MMA commit
  uint64_t accfull[2];          // MMA commit
  uint64_t accempty[2];         // 4 epilogue warps
  uint32_t tmem_base;
  int abort;
};

// x rounded to TF32 (round to nearest, ties away), as an FP32 value whose low
// 13 mantissa bits are zero.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Byte offset of element kk (< 32) of row `row` in a K-major tile of
// 128-byte rows with the 128-byte swizzle (16-byte group kk / 4 stored at
// group (kk / 4) xor (row mod 8)); the tile starts on a 1024-byte boundary.
__device__ __forceinline__ uint32_t sw128_off(int row, int kk) {
  return (uint32_t)row * 128u + ((uint32_t)((kk >> 2) ^ (row & 7)) << 4) + (uint32_t)(kk & 3) * 4u;
}

__device__ __forceinline__ void mbar_expect_tx_only(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(tc::smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"((uint64_t)src), "r"(bytes), "r"(tc::smem_u32(bar))
               : "memory");
}

// Images of B0 and B1 (FP64, K x N row-major): for product g, part h (0 hi,
// 1 lo) and chunk c, the Np x 32 tile B^T[n][c 32 + kk] in its swizzled
// layout at img + ((g 2 + h) nk + c) Np 128 bytes; entries beyond K or N are
// zero.
__global__ void extrap_bimg_kernel(const double* __restrict__ B0, const double* __restrict__ B1, int K, int N, int nk,
                                   int Np, uint8_t* __restrict__ img) {
  const long long per = (long long)nk * Np * 32;
  const long long total = 2 * per;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int g = (int)(e / per);
    long long r = e - (long long)g * per;
    const int c = (int)(r / ((long long)Np * 32));
    r -= (long long)c * Np * 32;
    const int n = (int)(r >> 5), kk = (int)(r & 31);
    const int kg = c * 32 + kk;
    const double* B = g ? B1 : B0;
    const float v = (kg < K && n < N) ? (float)B[(size_t)kg * N + n] : 0.f;
    const float hi = tf32_round(v);
    const uint32_t off = sw128_off(n, kk);
    *(float*)(img + ((size_t)(g * 2 + 0) * nk + c) * Np * 128 + off) = hi;
    *(float*)(img + ((size_t)(g * 2 + 1) * nk + c) * Np * 128 + off) = v - hi;
  }
}

__host__ __device__ constexpr size_t xstage_bytes(int Np) { return (size_t)2 * kXBM * 128 + (size_t)2 * Np * 128; }

__global__ void __launch_bounds__(kXThreads, 1)
    tc_extrap_kernel(const float* __restrict__ X, long long M, int K, int N, int Np, int nk, int tcols,
                     const uint8_t* __restrict__ bimg_hi, const uint8_t* __restrict__ bimg_lo, float* __restrict__ out,
                     double* __restrict__ part, int units, int* err) {
  extern __shared__ uint8_t smem_raw[];
  __shared__ XBars bars;
  __shared__ double colred[4][256];
  uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const size_t sb = xstage_bytes(Np);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kXStages; ++i) {
      tc::mbar_init(&bars.full[i], kXProd);
      tc::mbar_init(&bars.empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(&bars.accfull[i], 1);
      tc::mbar_init(&bars.accempty[i], 4);
    }
    bars.abort = 0;
    tc::fence_barrier_init();
  }
  if (warp == kXTmemWarp) tc::tmem_alloc(&bars.tmem_base, (uint32_t)(2 * tcols));
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  volatile int* abort = &bars.abort;
  const int u0 = (int)((long long)units * blockIdx.x / gridDim.x);
  const int u1 = (int)((long long)units * (blockIdx.x + 1) / gridDim.x);
  if (warp < 4) {
    // ---- producers: warp w stages rows 32 w .. 32 w + 31 of each tile
    const uint32_t bbytes = (uint32_t)(Np * 128);
    float v[32], nv[32];
    auto load = [&](float(&dst)[32], int u, int c) {
      const long long r0 = (long long)u * kXBM + warp * 32;
      const int kg = c * 32 + lane;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const long long gm = r0 + i;
        dst[i] = (gm < M && kg < K) ? __ldg(X + gm * K + kg) : 0.f;
      }
    };
    if (u0 < u1) load(v, u0, 0);
    int s = 0;
    uint32_t ph = 0;
    bool fail = false;
    for (int u = u0; u < u1 && !fail; ++u) {
      for (int c = 0; c < nk; ++c) {
        // the next chunk's loads are in flight while this one is written
        const bool more = c + 1 < nk || u + 1 < u1;
        if (more) load(nv, c + 1 < nk ? u : u + 1, c + 1 < nk ? c + 1 : 0);
        if (!tc::mbar_wait(&bars.empty[s], ph ^ 1, abort)) {
          fail = true;
          break;
        }
        uint8_t* st = base + (size_t)s * sb;
        if (threadIdx.x == 0) {
          mbar_expect_tx_only(&bars.full[s], 2 * bbytes);
          bulk_g2s(st + 2 * kXBM * 128, bimg_hi + (size_t)c * bbytes, bbytes, &bars.full[s]);
          bulk_g2s(st + 2 * kXBM * 128 + bbytes, bimg_lo + (size_t)c * bbytes, bbytes, &bars.full[s]);
        }
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int row = warp * 32 + i;
          const float hi = tf32_round(v[i]);
          const uint32_t off = sw128_off(row, lane);
          *(float*)(st + off) = hi;
          *(float*)(st + kXBM * 128 + off) = v[i] - hi;
        }
        // generic-proxy writes -> visible to the tensor core (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        tc::mbar_arrive(&bars.full[s]);
        if (more) {
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = nv[i];
        }
        if (++s == kXStages) {
          s = 0;
          ph ^= 1;
        }
      }
    }
  } else if (warp == kXMmaWarp) {
    // ---- MMA issuer
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(true, kXBM, Np);
      const uint32_t tbase = bars.tmem_base;
      int s = 0, ab = 0;
      uint32_t ph = 0, accph[2] = {0, 0};
      bool fail = false;
      for (int u = u0; u < u1 && !fail; ++u) {
        if (!tc::mbar_wait(&bars.accempty[ab], accph[ab] ^ 1, abort)) break;
        tc::fence_after_sync();
        const uint32_t dt = tbase + (uint32_t)(ab * tcols);
        for (int c = 0; c < nk; ++c) {
          if (!tc::mbar_wait(&bars.full[s], ph, abort)) {
            fail = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t st = tc::smem_u32(base + (size_t)s * sb);
          const uint32_t ahi = st, alo = st + kXBM * 128, bhi = st + 2 * kXBM * 128, blo = bhi + (uint32_t)(Np * 128);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            tc::mma<true>(dt, tc::sw128_desc(ahi + kk * 32), tc::sw128_desc(bhi + kk * 32), idesc,
                          (c > 0 || kk > 0) ? 1u : 0u);
            tc::mma<true>(dt, tc::sw128_desc(ahi + kk * 32), tc::sw128_desc(blo + kk * 32), idesc, 1u);
            tc::mma<true>(dt, tc::sw128_desc(alo + kk * 32), tc::sw128_desc(bhi + kk * 32), idesc, 1u);
          }
          tc::mma_commit(&bars.empty[s]);
          if (++s == kXStages) {
            s = 0;
            ph ^= 1;
          }
        }
        if (fail) break;
        tc::mma_commit(&bars.accfull[ab]);
        accph[ab] ^= 1;
        ab ^= 1;
      }
    }
  } else if (warp >= kXEpi0 && warp < kXEpi0 + 4) {
    // ---- epilogue: warp kXEpi0 + q reads TMEM lanes 32 q .. 32 q + 31
    const int q = warp - kXEpi0;
    const int row = q * 32 + lane;
    const uint32_t tbase = bars.tmem_base;
    const bool vec = (N & 3) == 0;
    int ab = 0;
    uint32_t accph[2] = {0, 0};
    for (int u = u0; u < u1; ++u) {
      tc::mbar_wait(&bars.accfull[ab], accph[ab], abort);
      // the four warps leave together (they share named barrier 1)
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (*abort) break;
      tc::fence_after_sync();
      const long long gm = (long long)u * kXBM + row;
      const bool valid = gm < M;
      for (int cb = 0; cb * 32 < N; ++cb) {
        float v[32];
        tc::tmem_ld32(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(ab * tcols + cb * 32), v);
        if (valid) {
          float* o = out + gm * N + cb * 32;
          if (vec && cb * 32 + 32 <= N) {
#pragma unroll
            for (int j = 0; j < 8; ++j)
              reinterpret_cast<float4*>(o)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j)
              if (cb * 32 + j < N) o[j] = v[j];
          }
        }
        // sums of squares over the warp's 32 rows: a halving exchange leaves
        // lane l with column cb 32 + l (16 + 8 + 4 + 2 + 1 shuffles)
        float sq[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) sq[j] = valid ? v[j] * v[j] : 0.f;
#pragma unroll
        for (int w = 16; w >= 1; w >>= 1) {
          const bool up = (lane & w) != 0;
#pragma unroll
          for (int i = 0; i < w; ++i) {
            const float send = up ? sq[i] : sq[i + w];
            const float keep = up ? sq[i + w] : sq[i];
            sq[i] = keep + __shfl_xor_sync(0xffffffffu, send, w);
          }
        }
        colred[q][cb * 32 + lane] = (double)sq[0];
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&bars.accempty[ab]);
      asm volatile("bar.sync 1, 128;" ::: "memory");
      if (q == 0)
        for (int col = lane; col < N; col += 32)
          part[(size_t)u * N + col] = ((colred[0][col] + colred[1][col]) + colred[2][col]) + colred[3][col];
      asm volatile("bar.sync 1, 128;" ::: "memory");
      accph[ab] ^= 1;
      ab ^= 1;
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (threadIdx.x == 0 && bars.abort && err) atomicOr(err, 4);
  if (warp == kXTmemWarp) {
    tc::fence_after_sync();
    tc::tmem_dealloc(bars.tmem_base, (uint32_t)(2 * tcols));
  }
}

struct XShape {
  int nk, Np, tcols;
};

XShape xshape(int k) {
  XShape s;
  s.nk = ceil_div(k, 32);
  s.Np = ceil_div(k, 16) * 16;
  s.tcols = 32;
  while (s.tcols < s.Np) s.tcols *= 2;
  return s;
}

cabs_status launch_one(const float* X, int64_t M, int k, const uint8_t* hi, const uint8_t* lo, float* out,
                       double* part, int* err, const char* name, cudaStream_t stream) {
  const XShape sh = xshape(k);
  const int units = ceil_div(M, kXBM);
  const int grid = std::max(1, std::min(units, sm_count()));
  const size_t smem = (size_t)kXStages * xstage_bytes(sh.Np) + 1024;
  cudaFuncSetAttribute(tc_extrap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  CABS_LAUNCH(stream, name,
              tc_extrap_kernel<<<grid, kXThreads, smem, stream>>>(X, M, k, k, sh.Np, sh.nk, sh.tcols, hi, lo, out,
                                                                   part, units, err));
  return CABS_OK;
}

}  // namespace

size_t tc_extrap_img_bytes(int k) {
  const XShape sh = xshape(k);
  return (size_t)4 * sh.nk * sh.Np * 128;
}

cabs_status launch_tc_extrap_pair(const float* C, int64_t m, const float* Rt, int64_t n, int k, const double* Vw,
                                  const double* Uw, float* out1, float* out2, double* part1, double* part2, void* img,
                                  int* status, cudaStream_t stream) {
  if (k < 1 || k > 256) {
    set_error("tensor-core extrapolation: k = %d outside 1..256", k);
    return CABS_EINVAL;
  }
  const XShape sh = xshape(k);
  uint8_t* im = (uint8_t*)img;
  const size_t one = (size_t)sh.nk * sh.Np * 128;
  const long long total = 2ll * sh.nk * sh.Np * 32;
  CABS_LAUNCH(stream, "extrap_bimg_kernel",
              extrap_bimg_kernel<<<std::max(1, (int)std::min<long long>(ceil_div(total, 256), 1024)), 256, 0, stream>>>(
                  Vw, Uw, k, k, sh.nk, sh.Np, im));
  CABS_TRY(launch_one(C, m, k, im, im + one, out1, part1, status, "tc_extrap_kernel(C V_w)", stream));
  CABS_TRY(launch_one(Rt, n, k, im + 2 * one, im + 3 * one, out2, part2, status, "tc_extrap_kernel(Rt U_w)", stream));
  return CABS_OK;
}

}  // namespace cabs
