// Step a9 -- relative Frobenius error |A - U diag(S) V^T|_F / |A|_F, the
// accuracy measure of Section 5.
//
// Exact (dense A): a fused tiled pass. Each CTA forms a 64 x 64 tile of
// A_hat = (U diag(S)) V^T from the k-wide factors in shared memory, reads the
// same tile of A once, and accumulates sum (a - a_hat)^2 and sum a^2 (per
// thread in the working precision, across threads in FP64).
// A is read exactly once; A_hat is never stored.
// Sampled (dense or implicit RBF): `samples` entries (i, j) drawn with
// replacement from Philox key (seed, 2), counter (t, 0, 0, 0): i = hi64(w0 m),
// j = hi64(w1 n); a_hat = sum_r U[i,r] S[r] V[j,r] in the working precision,
// squares summed in FP64.
// Per-CTA partial sums are added in a fixed order (deterministic).
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace cabs {
namespace {

constexpr int kRT = 64, kRK = 16;

template <typename T>
__global__ void __launch_bounds__(256) residual_dense_kernel(const T* __restrict__ U, const double* __restrict__ S,
                                                             const T* __restrict__ V, int k, const void* A,
                                                             int a_f64, long long lda, long long m, long long n,
                                                             double* __restrict__ part) {
  __shared__ __align__(16) T Us[kRK][kRT + 4];
  __shared__ __align__(16) T Vs[kRK][kRT + 4];
  __shared__ double red[2][8];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long i0 = (long long)blockIdx.y * kRT, j0 = (long long)blockIdx.x * kRT;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int r0 = 0; r0 < k; r0 += kRK) {
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
    for (int kk = 0; kk < kRK; ++kk) {
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
  // T-precision sums over this thread's 16 entries, FP64 across threads
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
  double num = (double)tn, den = (double)td;
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
    const size_t b = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    part[2 * b] = s0;
    part[2 * b + 1] = s1;
  }
}

template <typename T>
__device__ __forceinline__ double entry_of(const cabs_source& src, long long i, long long j) {
  if (src.kind == CABS_SRC_DENSE) {
    return src.a_is_f64 ? ((const double*)src.A)[i * src.lda + j]
                        : (double)((const float*)src.A)[i * src.lda + j];
  }
  const int d = src.d;
  T acc = T(0);
  for (int q = 0; q < d; ++q) {
    const T diff = (T)src.X[i * d + q] - (T)src.Y[j * d + q];
    acc = fma(diff, diff, acc);
  }
  const T c = (T)(1.0 / (2.0 * (double)src.sigma * (double)src.sigma));
  return (double)dev_exp<T>(-acc * c);
}

template <typename T>
__global__ void __launch_bounds__(256) residual_sampled_kernel(cabs_source src, long long m, long long n, int k,
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
    // a_hat in the working precision (FP64 arithmetic is 1/64 of FP32 here)
    const T a = (T)entry_of<T>(src, i, j);
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

__global__ void pair_reduce_kernel(const double* __restrict__ part, long long nb, double* __restrict__ out) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  for (long long i = threadIdx.x; i < nb; i += blockDim.x) {
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
    out[0] = s0[0];
    out[1] = s1[0];
  }
}

long long sampled_blocks(long long samples) {
  return std::max<long long>(1, std::min<long long>((samples + 255) / 256, (long long)sm_count() * 8));
}

long long dense_blocks(int64_t m, int64_t n) { return (long long)ceil_div(m, kRT) * ceil_div(n, kRT); }

template <typename T>
cabs_status error_typed(const cabs_source& src, int64_t m, int64_t n, int k, const T* U, const double* S, const T* V,
                        int64_t samples, uint64_t seed, void* ws, size_t ws_bytes, double* out2,
                        cudaStream_t stream) {
  const long long nb = samples > 0 ? sampled_blocks(samples) : dense_blocks(m, n);
  if ((size_t)nb * 16 > ws_bytes) {
    set_error("error workspace too small: need %lld bytes", nb * 16);
    return CABS_ENOMEM;
  }
  double* part = (double*)ws;
  if (samples > 0) {
    CABS_LAUNCH(stream, "residual_sampled_kernel", residual_sampled_kernel<T><<<(int)nb, 256, 0, stream>>>(src, m, n, k, U, S, V, samples, seed, part));
  } else {
    dim3 grid(ceil_div(n, kRT), ceil_div(m, kRT));
    CABS_LAUNCH(stream, "residual_dense_kernel", residual_dense_kernel<T><<<grid, 256, 0, stream>>>(U, S, V, k, src.A, src.a_is_f64, src.lda, m, n, part));
  }
  CABS_LAUNCH(stream, "pair_reduce_kernel", pair_reduce_kernel<<<1, 256, 0, stream>>>(part, nb, out2));
  return CABS_OK;
}

}  // namespace

// The tensor-core residual streams A by TMA: rows must start on 16-byte
// boundaries (lda a multiple of 4 floats, A 16-byte aligned).
static bool use_tc_residual(const cabs_source& src, int64_t samples, int prec) {
  return samples == 0 && src.kind == CABS_SRC_DENSE && !src.a_is_f64 &&
         (prec == CABS_PREC_TF32 || prec == CABS_PREC_BF16) && (src.lda & 3) == 0 &&
         ((uintptr_t)src.A & 15) == 0;
}

size_t error_ws_bytes(const cabs_source& src, int64_t m, int64_t n, int k, int64_t samples, int prec) {
  if (use_tc_residual(src, samples, prec)) return tc_residual_ws_bytes(m, n, k, prec == CABS_PREC_TF32);
  const long long nb = samples > 0 ? sampled_blocks(samples) : dense_blocks(m, n);
  return align256((size_t)nb * 16) + 256;
}

cabs_status launch_error(const cabs_source& src, int64_t m, int64_t n, int k, bool elem_f64, int prec,
                         const void* U, const double* S, const void* V, int64_t samples, uint64_t seed, void* ws,
                         size_t ws_bytes, double* d_out2, cudaStream_t stream) {
  if (use_tc_residual(src, samples, prec))
    return launch_tc_residual(src, m, n, k, prec == CABS_PREC_TF32, (const float*)U, S, (const float*)V, ws, ws_bytes,
                              d_out2, stream);
  if (elem_f64)
    return error_typed<double>(src, m, n, k, (const double*)U, S, (const double*)V, samples, seed, ws, ws_bytes,
                               d_out2, stream);
  return error_typed<float>(src, m, n, k, (const float*)U, S, (const float*)V, samples, seed, ws, ws_bytes, d_out2,
                            stream);
}

}  // namespace cabs
