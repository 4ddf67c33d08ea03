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
// Exact (sparse A in compressed rows): the identity
//   |A - L|_F^2 = |A|_F^2 - 2 sum_{stored (i,j)} a_ij L_ij + |L|_F^2,
//   |L|_F^2 = sum_{p,q} S_p S_q (U^T U)_pq (V^T V)_pq,   L = U diag(S) V^T,
// costs O(nnz k + (m + n) k^2) instead of O(m n k): one warp per row forms
// L_ij at the row's stored entries only, and the two Gram matrices come from
// the tall Gram kernel. The three terms are FP64 sums (the cross term's dot
// products in the working precision).
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
  if (src.kind == CABS_SRC_CSR) {
    long long lo, hi;
    csr_row_range((const long long*)src.row_ptr, src.nnz, i, lo, hi);
    const long long e = csr_find(src.col_idx, lo, hi, (int)j);
    if (e < 0) return 0.0;
    return src.a_is_f64 ? ((const double*)src.A)[e] : (double)((const float*)src.A)[e];
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

// Sparse exact error, stored entries: per CTA, sum a^2 and sum a L_ij. The
// stored entries are split evenly over the warps (row degrees can follow a
// power law, so rows would not balance); a warp walks the rows its range
// touches, holding U_i diag(S) in registers (k / 32 per lane), reads row j of
// V coalesced for each entry and reduces the dot product across its lanes,
// four entries at a time.
template <typename T, typename Tin>
__global__ void __launch_bounds__(256) csr_cross_kernel(const long long* __restrict__ row_ptr,
                                                        const int* __restrict__ col_idx, const Tin* __restrict__ vals,
                                                        long long nnz, long long m, long long n, int k,
                                                        const T* __restrict__ U, const double* __restrict__ S,
                                                        const T* __restrict__ V, double* __restrict__ part) {
  constexpr int kPer = CABS_MAX_K / 32;
  __shared__ double red[2][8];
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const long long nwarps = (long long)gridDim.x * 8, gw = (long long)blockIdx.x * 8 + wi;
  const long long per = (nnz + nwarps - 1) / nwarps;
  const long long e_lo = min(nnz, gw * per), e_hi = min(nnz, e_lo + per);
  double sq = 0.0, cr = 0.0;
  if (e_lo < e_hi) {
    // first row whose range reaches past e_lo (row_ptr clamped to [0, nnz])
    long long lo = 0, hi = m;
    while (lo < hi) {
      const long long mid = (lo + hi) >> 1;
      if (min(max(row_ptr[mid + 1], 0ll), nnz) <= e_lo) lo = mid + 1;
      else hi = mid;
    }
    for (long long i = lo; i < m; ++i) {
      long long r0, r1;
      csr_row_range(row_ptr, nnz, i, r0, r1);
      r0 = max(r0, e_lo);
      r1 = min(r1, e_hi);
      if (r0 >= e_hi) break;
      if (r0 >= r1) continue;
      T us[kPer];
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int r = lane + 32 * t;
        us[t] = r < k ? U[i * k + r] * (T)S[r] : T(0);
      }
      for (long long e = r0; e < r1; e += 4) {
        int js[4];
        double as[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool in = e + u < r1;
          const int j = in ? col_idx[e + u] : -1;
          js[u] = (j >= 0 && j < n) ? j : -1;
          as[u] = in ? (double)vals[e + u] : 0.0;
        }
        T dots[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          T dot = T(0);
          if (js[u] >= 0) {
            const T* v = V + (long long)js[u] * k;
#pragma unroll
            for (int t = 0; t < kPer; ++t) {
              const int r = lane + 32 * t;
              if (r < k) dot = fma(us[t], v[r], dot);
            }
          }
          dots[u] = dot;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
          for (int u = 0; u < 4; ++u) dots[u] += __shfl_xor_sync(0xffffffffu, dots[u], off);
        if (lane == 0) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            sq += as[u] * as[u];
            cr += as[u] * (double)dots[u];
          }
        }
      }
    }
  }
  sq = warp_sum(sq);
  cr = warp_sum(cr);
  if (lane == 0) {
    red[0][wi] = sq;
    red[1][wi] = cr;
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

// (num, den) = (|A|^2 - 2 cross + sum_pq S_p S_q Gu_pq Gv_pq, |A|^2) from the
// reduced (|A|^2, cross) in out2 and the Gram matrices. One CTA.
__global__ void __launch_bounds__(256) csr_finish_kernel(int k, const double* __restrict__ S,
                                                         const double* __restrict__ Gu, const double* __restrict__ Gv,
                                                         double* __restrict__ out2) {
  __shared__ double red[256];
  double l2 = 0.0;
  for (long long e = threadIdx.x; e < (long long)k * k; e += blockDim.x) {
    const int p = (int)(e / k), q = (int)(e - (long long)p * k);
    l2 += S[p] * S[q] * Gu[e] * Gv[e];
  }
  red[threadIdx.x] = l2;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double a2 = out2[0], cross = out2[1];
    out2[0] = fmax(a2 - 2.0 * cross + red[0], 0.0);
    out2[1] = a2;
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

long long csr_blocks(int64_t m) {
  return std::max<long long>(1, std::min<long long>((m + 7) / 8, (long long)sm_count() * 8));
}

// Workspace of the sparse exact error: partials, two Gram matrices, Gram scratch.
size_t csr_error_ws_bytes(int64_t m, int64_t n, int k, bool f64) {
  return align256((size_t)csr_blocks(m) * 16) + 2 * align256((size_t)k * k * 8) +
         std::max(gram_ws_bytes(m, k, f64), gram_ws_bytes(n, k, f64));
}

template <typename T>
cabs_status csr_error_typed(const cabs_source& src, int64_t m, int64_t n, int k, const T* U, const double* S,
                            const T* V, void* ws, size_t ws_bytes, double* out2, cudaStream_t stream) {
  if (csr_error_ws_bytes(m, n, k, sizeof(T) == 8) > ws_bytes) {
    set_error("error workspace too small for the sparse exact error");
    return CABS_ENOMEM;
  }
  Carve cv(ws, ws_bytes);
  const long long nb = csr_blocks(m);
  double* part = cv.take<double>((size_t)nb * 2);
  double* Gu = cv.take<double>((size_t)k * k);
  double* Gv = cv.take<double>((size_t)k * k);
  void* gpart = cv.take<char>(std::max(gram_ws_bytes(m, k, sizeof(T) == 8), gram_ws_bytes(n, k, sizeof(T) == 8)));
  const long long* rp = (const long long*)src.row_ptr;
  if (src.a_is_f64)
    CABS_LAUNCH(stream, "csr_cross_kernel",
                csr_cross_kernel<T, double><<<(int)nb, 256, 0, stream>>>(rp, src.col_idx, (const double*)src.A,
                                                                         src.nnz, m, n, k, U, S, V, part));
  else
    CABS_LAUNCH(stream, "csr_cross_kernel",
                csr_cross_kernel<T, float><<<(int)nb, 256, 0, stream>>>(rp, src.col_idx, (const float*)src.A, src.nnz,
                                                                        m, n, k, U, S, V, part));
  CABS_LAUNCH(stream, "pair_reduce_kernel", pair_reduce_kernel<<<1, 256, 0, stream>>>(part, nb, out2));
  CABS_TRY(launch_gram(U, m, k, sizeof(T) == 8, gpart, Gu, stream));
  CABS_TRY(launch_gram(V, n, k, sizeof(T) == 8, gpart, Gv, stream));
  CABS_LAUNCH(stream, "csr_finish_kernel", csr_finish_kernel<<<1, 256, 0, stream>>>(k, S, Gu, Gv, out2));
  return CABS_OK;
}

template <typename T>
cabs_status error_typed(const cabs_source& src, int64_t m, int64_t n, int k, const T* U, const double* S, const T* V,
                        int64_t samples, uint64_t seed, void* ws, size_t ws_bytes, double* out2,
                        cudaStream_t stream) {
  if (samples == 0 && src.kind == CABS_SRC_CSR) return csr_error_typed<T>(src, m, n, k, U, S, V, ws, ws_bytes, out2, stream);
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
  if (samples == 0 && src.kind == CABS_SRC_CSR) return csr_error_ws_bytes(m, n, k, prec == CABS_PREC_FP64) + 256;
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
