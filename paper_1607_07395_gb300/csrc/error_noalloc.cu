// cabs_error_noalloc: the relative Frobenius error of a sketch without any
// device allocation by the library or the caller beyond the inputs.
//
// Some callers cannot allocate device memory at the point where they want
// the error: code running inside another framework's memory pool that
// forbids cudaMalloc/cudaFree during a step, or embedded callers that
// reserve all device memory up front and have no workspace left to hand out.
// For them this variant keeps its scratch (per-CTA partial sums and the two
// final sums) in one file-scope device array of fixed size, which every GPU
// that loads libcabs holds until the process exits.
//
// Arithmetic: the products U diag(S) V^T are FP64 in FP64 mode and FP32
// CUDA-core products in the FP32, TF32 and BF16 modes. cabs_error takes the
// tensor-core residual for TF32 / BF16 on a dense FP32 A (TF32 / BF16
// operands); there this variant returns the FP32-mode value of the same
// factors instead, within 1e-3 relative of cabs_error's.
//
// Limits: the exact (dense) error uses one CTA per 64-row block of A, so
// m <= 64 * kNoAllocMaxBlocks = 1,048,576 rows; the sampled error uses at
// most kNoAllocMaxBlocks CTAs for any sample count. Larger m is rejected
// with CABS_EINVAL before anything is launched.
//
// Sharing: every call uses the same array and leaves its contents behind.
// Each call overwrites every slot it reads, so nothing needs clearing, but
// two calls whose kernels overlap on the GPU (different streams, or
// different host threads) race on the array and may return wrong values.
//
// Set-up: the array's device address is looked up once per device, with
// that device current (cudaGetSymbolAddress), on the first call made on that
// device; make that first call before any CUDA stream capture begins.
#include <cmath>
#include <mutex>

#include "api_internal.cuh"
#include "common.cuh"
#include "profile.cuh"

namespace cabs {
namespace {

constexpr int kNoAllocMaxBlocks = 16384;
constexpr int kTile = 64, kTileK = 16;

// [0, 2 * kNoAllocMaxBlocks): per-CTA (num, den); the last two: the totals.
static __device__ __align__(256) double g_error_scratch[2 * kNoAllocMaxBlocks + 2];

std::mutex g_sym_mu;
double* g_sym_ptr[64] = {nullptr};

cabs_status scratch_address(int dev, double** out) {
  if (dev < 0 || dev >= 64) {
    set_error("device index %d out of range for the no-allocation scratch", dev);
    return CABS_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_sym_mu);
  if (!g_sym_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_error_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      set_error("cudaGetSymbolAddress(no-allocation scratch) failed: %s", cudaGetErrorString(e));
      return CABS_ECUDA;
    }
    g_sym_ptr[dev] = (double*)p;
  }
  *out = g_sym_ptr[dev];
  return CABS_OK;
}

// One CTA per 64-row block of A: walks every 64 x 64 column tile of its rows,
// forms the tile of (U diag(S)) V^T as the exact-error kernel does, and sums
// (a - a_hat)^2 and a^2 over all of them into its own pair of slots.
template <typename T>
__global__ void __launch_bounds__(256) rowblock_error_kernel(const T* __restrict__ U, const double* __restrict__ S,
                                                             const T* __restrict__ V, int k, const void* A, int a_f64,
                                                             long long lda, long long m, long long n,
                                                             double* __restrict__ part) {
  __shared__ __align__(16) T Us[kTileK][kTile + 4];
  __shared__ __align__(16) T Vs[kTileK][kTile + 4];
  __shared__ double red[2][8];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long i0 = (long long)blockIdx.x * kTile;
  double num = 0.0, den = 0.0;
  for (long long j0 = 0; j0 < n; j0 += kTile) {
    T acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
    for (int r0 = 0; r0 < k; r0 += kTileK) {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int idx = tid + 256 * e;
        const int row = idx >> 4, c = idx & 15;
        const int r = r0 + c;
        const long long gi = i0 + row, gj = j0 + row;
        Us[c][row] = (gi < m && r < k) ? (T)((double)U[gi * k + r] * S[r]) : T(0);
        Vs[c][row] = (gj < n && r < k) ? V[gj * k + r] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kTileK; ++kk) {
        T a[4], b[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) a[x] = Us[kk][ty * 4 + x];
#pragma unroll
        for (int y = 0; y < 4; ++y) b[y] = Vs[kk][tx * 4 + y];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
      }
      __syncthreads();
    }
    T tn = T(0), td = T(0);
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const long long gi = i0 + ty * 4 + x;
      if (gi >= m) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const long long gj = j0 + tx * 4 + y;
        if (gj >= n) continue;
        const T a = a_f64 ? (T)((const double*)A)[gi * lda + gj] : (T)((const float*)A)[gi * lda + gj];
        const T dlt = a - acc[x][y];
        tn = fma(dlt, dlt, tn);
        td = fma(a, a, td);
      }
    }
    num += (double)tn;
    den += (double)td;
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = num;
    red[1][tid >> 5] = den;
  }
  __syncthreads();
  if (tid == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < 8; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

template <typename T>
__device__ __forceinline__ double noalloc_entry(const cabs_source& src, long long i, long long j) {
  if (src.kind == CABS_SRC_DENSE)
    return src.a_is_f64 ? ((const double*)src.A)[i * src.lda + j] : (double)((const float*)src.A)[i * src.lda + j];
  if (src.kind == CABS_SRC_CSR) {
    long long lo, hi;
    csr_row_range((const long long*)src.row_ptr, src.nnz, i, lo, hi);
    const long long e = csr_find(src.col_idx, lo, hi, (int)j);
    if (e < 0) return 0.0;
    return src.a_is_f64 ? ((const double*)src.A)[e] : (double)((const float*)src.A)[e];
  }
  T acc = T(0);
  for (int q = 0; q < src.d; ++q) {
    const T diff = (T)src.X[i * src.d + q] - (T)src.Y[j * src.d + q];
    acc = fma(diff, diff, acc);
  }
  const T c = (T)(1.0 / (2.0 * (double)src.sigma * (double)src.sigma));
  return (double)dev_exp<T>(-acc * c);
}

// Sampled entries (Philox key (seed, 2), counter (t, 0, 0, 0)), grid-stride.
template <typename T>
__global__ void __launch_bounds__(256) sampled_error_kernel(cabs_source src, long long m, long long n, int k,
                                                            const T* __restrict__ U, const double* __restrict__ S,
                                                            const T* __restrict__ V, long long samples,
                                                            unsigned long long seed, double* __restrict__ part) {
  __shared__ double red[2][8];
  double num = 0.0, den = 0.0;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < samples;
       t += (long long)gridDim.x * blockDim.x) {
    const U64x4 r = philox4x64_10((uint64_t)t, 0, 0, 0, seed, 2);
    const long long i = (long long)mulhi64(r.v[0], (uint64_t)m);
    const long long j = (long long)mulhi64(r.v[1], (uint64_t)n);
    const T a = (T)noalloc_entry<T>(src, i, j);
    T ah = T(0);
    for (int c = 0; c < k; ++c) ah = fma(U[i * k + c] * (T)S[c], V[j * k + c], ah);
    const T dl = a - ah;
    num += (double)(dl * dl);
    den += (double)(a * a);
  }
  num = warp_sum(num);
  den = warp_sum(den);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = num;
    red[1][threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s0 = 0.0, s1 = 0.0;
    for (int w = 0; w < 8; ++w) {
      s0 += red[0][w];
      s1 += red[1][w];
    }
    part[2 * blockIdx.x] = s0;
    part[2 * blockIdx.x + 1] = s1;
  }
}

// Sums the per-CTA pairs in a fixed order into the last two slots.
__global__ void noalloc_total_kernel(double* __restrict__ scratch, int nb) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    a += scratch[2 * i];
    b += scratch[2 * i + 1];
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
    scratch[2 * kNoAllocMaxBlocks] = s0[0];
    scratch[2 * kNoAllocMaxBlocks + 1] = s1[0];
  }
}

template <typename T>
cabs_status noalloc_typed(const cabs_source& src, int64_t m, int64_t n, int k, const T* U, const double* S,
                          const T* V, int64_t samples, uint64_t seed, double* scratch, cudaStream_t stream) {
  int nb;
  if (samples > 0) {
    nb = (int)std::max<long long>(1, std::min<long long>((samples + 255) / 256, (long long)sm_count() * 8));
    nb = std::min(nb, kNoAllocMaxBlocks);
    CABS_LAUNCH(stream, "sampled_error_kernel(noalloc)",
                sampled_error_kernel<T><<<nb, 256, 0, stream>>>(src, m, n, k, U, S, V, samples, seed, scratch));
  } else {
    nb = ceil_div(m, kTile);
    CABS_LAUNCH(stream, "rowblock_error_kernel(noalloc)",
                rowblock_error_kernel<T><<<nb, 256, 0, stream>>>(U, S, V, k, src.A, src.a_is_f64, src.lda, m, n,
                                                                 scratch));
  }
  CABS_LAUNCH(stream, "noalloc_total_kernel", noalloc_total_kernel<<<1, 256, 0, stream>>>(scratch, nb));
  return CABS_OK;
}

}  // namespace
}  // namespace cabs

using namespace cabs;

extern "C" cabs_status cabs_error_noalloc(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p,
                                          const cabs_result* res, int64_t samples, uint64_t seed, cabs_stream stream,
                                          double* rel_fro) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && rel_fro != nullptr, "ctx and rel_fro must be non-NULL");
  CABS_TRY(validate_params(p));
  CABS_TRY(validate_source(src, p->m, p->n));
  CABS_REQUIRE(res != nullptr && res->U && res->S && res->V, "result U, S, V must be set");
  CABS_REQUIRE(samples >= 0, "samples must be >= 0");
  CABS_REQUIRE(samples > 0 || src->kind == CABS_SRC_DENSE,
               "the exact error without a workspace needs a dense source (cabs_error takes CSR too)");
  CABS_REQUIRE(samples > 0 || p->m <= (int64_t)kTile * kNoAllocMaxBlocks,
               "the no-allocation exact error supports m <= %d rows (its fixed scratch holds %d row blocks); "
               "got m = %lld", kTile * kNoAllocMaxBlocks, kNoAllocMaxBlocks, (long long)p->m);
  DeviceGuard g(ctx->device);
  if (!g.ok) {
    set_error("cannot select CUDA device %d", ctx->device);
    return CABS_ECUDA;
  }
  double* scratch = nullptr;
  CABS_TRY(scratch_address(ctx->device, &scratch));
  cudaStream_t s = (cudaStream_t)stream;
  const bool f64 = p->prec == CABS_PREC_FP64;
  const cabs_status st =
      f64 ? noalloc_typed<double>(*src, p->m, p->n, p->k2, (const double*)res->U, res->S, (const double*)res->V,
                                  samples, seed, scratch, s)
          : noalloc_typed<float>(*src, p->m, p->n, p->k2, (const float*)res->U, res->S, (const float*)res->V, samples,
                                 seed, scratch, s);
  if (st != CABS_OK) return st;
  double h[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(h, scratch + 2 * kNoAllocMaxBlocks, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return check_cuda("cabs_error_noalloc readback");
  *rel_fro = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
  return CABS_OK;
}
