// Steps a2 / a7 -- the bilateral gathers of Algorithm 2 (steps 1 and 3):
//   C  = A[:, J]      m x kc, row-major (one output row per row of A)
//   Rt = A[I, :]^T    n x kr, row-major (R kept transposed, as in the proof of Theorem 1)
//   W  = A[I, J]      kr x kc, FP64, taken from C so that W == C[I, :] bit for bit
//
// Dense A (row-major, lda): the column gather reads one element of every
// selected column in each row of A; those are scattered 4- or 8-byte reads,
// one DRAM sector each, so the kernel keeps many independent loads in flight
// per thread (several rows x up to 8 columns per lane). The row gather reads
// k contiguous rows with coalesced loads and transposes them through a
// padded shared-memory tile so the n x k output is written coalesced.
//
// Sparse A in compressed rows (the sparse inputs of Table 1): C is filled
// one warp per row, each lane binary-searching the row's sorted column
// indices for its selected columns (absent entries are zero); Rt is zeroed
// and then each selected row scatters its stored entries into its column of
// Rt. Both read the stored value itself, so W == C[I, :] == Rt[J, :]^T.
//
// Implicit RBF A[i, j] = exp(-|x_i - y_j|^2 / 2 sigma^2): the same outputs
// are generated on the fly (the entries are never stored). C uses points X
// against the selected Y rows and Rt uses Y against the selected X rows; the
// arithmetic is identical up to the sign of each difference, so
// Rt[J_t, p] == C[I_p, t] bit for bit.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace cabs {
namespace {

constexpr int kGatherThreads = 256;
constexpr int kRowsPerWarp = 4;
constexpr int kMaxColsPerLane = CABS_MAX_K / 32;

// kRows rows per warp (the launch shape: loads in flight per thread).
template <typename Tin, typename Tout, int kRows = kRowsPerWarp>
__global__ void __launch_bounds__(kGatherThreads) gather_cols_kernel(const Tin* __restrict__ A, long long lda,
                                                                     long long m, long long n,
                                                                     const int* __restrict__ cols, int kc,
                                                                     Tout* __restrict__ C) {
  __shared__ int cs[CABS_MAX_K];
  for (int t = threadIdx.x; t < kc; t += blockDim.x) cs[t] = (int)min(max((long long)cols[t], 0ll), n - 1);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  int col[kMaxColsPerLane];
#pragma unroll
  for (int q = 0; q < kMaxColsPerLane; ++q) {
    const int t = lane + 32 * q;
    col[q] = t < kc ? cs[t] : 0;
  }
  for (long long i0 = warp * kRows; i0 < m; i0 += nwarps * kRows) {
    Tin v[kRows][kMaxColsPerLane];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const long long i = i0 + r;
      const Tin* row = A + (i < m ? i : 0) * lda;
#pragma unroll
      for (int q = 0; q < kMaxColsPerLane; ++q) {
        const int t = lane + 32 * q;
        v[r][q] = (i < m && t < kc) ? __ldg(row + col[q]) : Tin(0);
      }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const long long i = i0 + r;
      if (i >= m) break;
      Tout* out = C + i * kc;
#pragma unroll
      for (int q = 0; q < kMaxColsPerLane; ++q) {
        const int t = lane + 32 * q;
        if (t < kc) out[t] = (Tout)v[r][q];
      }
    }
  }
}

constexpr int kTileP = 32;   // sampled rows per tile
constexpr int kTileJ = 128;  // columns of A per tile

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kGatherThreads) gather_rows_t_kernel(const Tin* __restrict__ A, long long lda,
                                                                       long long m, long long n,
                                                                       const int* __restrict__ rows, int kr,
                                                                       Tout* __restrict__ Rt) {
  __shared__ Tout tile[kTileP][kTileJ + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int p0 = blockIdx.y * kTileP;
  for (long long j0 = (long long)blockIdx.x * kTileJ; j0 < n; j0 += (long long)gridDim.x * kTileJ) {
#pragma unroll
    for (int s = 0; s < kTileP / 8; ++s) {
      const int pp = w + 8 * s;
      const int p = p0 + pp;
      const Tin* src = p < kr ? A + min(max((long long)rows[p], 0ll), m - 1) * lda : nullptr;
#pragma unroll
      for (int q = 0; q < kTileJ / 32; ++q) {
        const long long j = j0 + lane + 32 * q;
        tile[pp][lane + 32 * q] = (p < kr && j < n) ? (Tout)__ldg(src + j) : Tout(0);
      }
    }
    __syncthreads();
    const int p = p0 + lane;
#pragma unroll 4
    for (int s = 0; s < kTileJ / 8; ++s) {
      const int jj = w + 8 * s;
      const long long j = j0 + jj;
      if (j < n && p < kr) Rt[j * kr + p] = tile[lane][jj];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void w_from_c_kernel(const T* __restrict__ C, long long m, int kc, const int* __restrict__ rows,
                                int kr, double* __restrict__ W) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kr * kc) return;
  const int p = idx / kc, t = idx - p * kc;
  W[idx] = (double)C[min(max((long long)rows[p], 0ll), m - 1) * kc + t];
}

// out[i, t] = exp(-|P_i - Q_{idx[t]}|^2 / (2 sigma^2)), T = working precision.
template <typename T>
__global__ void __launch_bounds__(kGatherThreads) rbf_block_kernel(const float* __restrict__ Pts, long long M,
                                                                   const float* __restrict__ Q, long long NQ,
                                                                   const int* __restrict__ idx, int kq, int d,
                                                                   double inv2s2, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* qs = (T*)smem_raw;  // kq x (d | 1) selected points, widened to T
  const int ld = d | 1;
  for (int e = threadIdx.x; e < kq * d; e += blockDim.x) {
    const int t = e / d, q = e - t * d;
    qs[t * ld + q] = (T)Q[min(max((long long)idx[t], 0ll), NQ - 1) * d + q];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long warp = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  const T c = (T)inv2s2;
  for (long long i = warp; i < M; i += nwarps) {
    const float* x = Pts + i * d;
    T acc[kMaxColsPerLane];
#pragma unroll
    for (int s = 0; s < kMaxColsPerLane; ++s) acc[s] = T(0);
    for (int q = 0; q < d; ++q) {
      const T xq = (T)__ldg(x + q);
#pragma unroll
      for (int s = 0; s < kMaxColsPerLane; ++s) {
        const int t = lane + 32 * s;
        if (t < kq) {
          const T diff = xq - qs[t * ld + q];
          acc[s] = fma(diff, diff, acc[s]);
        }
      }
    }
#pragma unroll
    for (int s = 0; s < kMaxColsPerLane; ++s) {
      const int t = lane + 32 * s;
      if (t < kq) out[i * kq + t] = dev_exp<T>(-acc[s] * c);
    }
  }
}

template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kGatherThreads) csr_cols_kernel(const long long* __restrict__ row_ptr,
                                                                  const int* __restrict__ col_idx,
                                                                  const Tin* __restrict__ vals, long long nnz,
                                                                  long long m, const int* __restrict__ cols, int kc,
                                                                  Tout* __restrict__ C) {
  __shared__ int cs[CABS_MAX_K];
  for (int t = threadIdx.x; t < kc; t += blockDim.x) cs[t] = cols[t];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < m; i += nwarps) {
    long long lo, hi;
    csr_row_range(row_ptr, nnz, i, lo, hi);
    for (int t = lane; t < kc; t += 32) {
      const long long e = csr_find(col_idx, lo, hi, cs[t]);
      C[i * kc + t] = e >= 0 ? (Tout)vals[e] : Tout(0);
    }
  }
}

// Rt[j, p] = A[rows[p], j]: one CTA per selected row p scatters its stored
// entries (Rt must be zero beforehand).
template <typename Tin, typename Tout>
__global__ void __launch_bounds__(kGatherThreads) csr_rows_t_kernel(const long long* __restrict__ row_ptr,
                                                                    const int* __restrict__ col_idx,
                                                                    const Tin* __restrict__ vals, long long nnz,
                                                                    long long m, long long n,
                                                                    const int* __restrict__ rows, int kr,
                                                                    Tout* __restrict__ Rt) {
  const int p = blockIdx.x;
  const long long i = min(max((long long)rows[p], 0ll), m - 1);
  long long lo, hi;
  csr_row_range(row_ptr, nnz, i, lo, hi);
  for (long long e = lo + threadIdx.x; e < hi; e += blockDim.x) {
    const int j = col_idx[e];
    if (j >= 0 && j < n) Rt[(long long)j * kr + p] = (Tout)vals[e];
  }
}

template <typename Tout>
__global__ void zero_kernel(Tout* __restrict__ x, long long count) {
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < count;
       e += (long long)gridDim.x * blockDim.x)
    x[e] = Tout(0);
}

template <typename Tout, int kRows>
cabs_status gather_cols_dense(const cabs_source& src, int64_t m, int64_t n, const int* cols, int kc, Tout* C,
                              cudaStream_t stream) {
  const int blocks = std::max(1, std::min(ceil_div(m, (kGatherThreads / 32) * kRows), sm_count() * 8));
  CABS_LAUNCH(stream, "gather_cols_kernel",
              if (src.a_is_f64)(gather_cols_kernel<double, Tout, kRows><<<blocks, kGatherThreads, 0, stream>>>(
                  (const double*)src.A, src.lda, m, n, cols, kc, C));
              else(gather_cols_kernel<float, Tout, kRows><<<blocks, kGatherThreads, 0, stream>>>(
                  (const float*)src.A, src.lda, m, n, cols, kc, C)));
  return CABS_OK;
}

template <typename Tout>
cabs_status gather_typed(const cabs_source& src, int64_t m, int64_t n, const int* rows, int kr, const int* cols,
                         int kc, Tout* C, Tout* Rt, double* W, cudaStream_t stream) {
  const int sms = sm_count();
  if (src.kind == CABS_SRC_DENSE) {
    if (C && kc > 0) {
      const int gr = current_tune().gather_rows;
      if (gr == 2)
        CABS_TRY((gather_cols_dense<Tout, 2>(src, m, n, cols, kc, C, stream)));
      else if (gr == 8)
        CABS_TRY((gather_cols_dense<Tout, 8>(src, m, n, cols, kc, C, stream)));
      else
        CABS_TRY((gather_cols_dense<Tout, kRowsPerWarp>(src, m, n, cols, kc, C, stream)));
    }
    if (Rt && kr > 0) {
      const int py = ceil_div(kr, kTileP);
      const int px = std::max(1, std::min(ceil_div(n, kTileJ), std::max(1, sms * 8 / py)));
      dim3 grid(px, py);
      CABS_LAUNCH(stream, "gather_rows_t_kernel",
                  if (src.a_is_f64) gather_rows_t_kernel<double, Tout><<<grid, kGatherThreads, 0, stream>>>(
                      (const double*)src.A, src.lda, m, n, rows, kr, Rt);
                  else gather_rows_t_kernel<float, Tout><<<grid, kGatherThreads, 0, stream>>>(
                      (const float*)src.A, src.lda, m, n, rows, kr, Rt));
    }
  } else if (src.kind == CABS_SRC_CSR) {
    const long long* rp = (const long long*)src.row_ptr;
    if (C && kc > 0) {
      const int blocks = std::max(1, std::min(ceil_div(m, kGatherThreads / 32), sms * 8));
      CABS_LAUNCH(stream, "csr_cols_kernel",
                  if (src.a_is_f64) csr_cols_kernel<double, Tout><<<blocks, kGatherThreads, 0, stream>>>(
                      rp, src.col_idx, (const double*)src.A, src.nnz, m, cols, kc, C);
                  else csr_cols_kernel<float, Tout><<<blocks, kGatherThreads, 0, stream>>>(
                      rp, src.col_idx, (const float*)src.A, src.nnz, m, cols, kc, C));
    }
    if (Rt && kr > 0) {
      const long long cnt = (long long)n * kr;
      CABS_LAUNCH(stream, "zero_kernel",
                  zero_kernel<Tout><<<(int)std::max<long long>(1, std::min<long long>((cnt + 255) / 256, sms * 8)), 256,
                                      0, stream>>>(Rt, cnt));
      CABS_LAUNCH(stream, "csr_rows_t_kernel",
                  if (src.a_is_f64) csr_rows_t_kernel<double, Tout><<<kr, kGatherThreads, 0, stream>>>(
                      rp, src.col_idx, (const double*)src.A, src.nnz, m, n, rows, kr, Rt);
                  else csr_rows_t_kernel<float, Tout><<<kr, kGatherThreads, 0, stream>>>(
                      rp, src.col_idx, (const float*)src.A, src.nnz, m, n, rows, kr, Rt));
    }
  } else {
    const double inv2s2 = 1.0 / (2.0 * (double)src.sigma * (double)src.sigma);
    const size_t smem = (size_t)std::max(kr, kc) * (src.d | 1) * sizeof(Tout);
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(rbf_block_kernel<Tout>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (C && kc > 0) {
      const int blocks = std::max(1, std::min(ceil_div(m, kGatherThreads / 32), sms * 8));
      CABS_LAUNCH(stream, "rbf_block_kernel(C)", rbf_block_kernel<Tout><<<blocks, kGatherThreads, smem, stream>>>(src.X, m, src.Y, n, cols, kc, src.d, inv2s2, C));
    }
    if (Rt && kr > 0) {
      const int blocks = std::max(1, std::min(ceil_div(n, kGatherThreads / 32), sms * 8));
      CABS_LAUNCH(stream, "rbf_block_kernel(Rt)", rbf_block_kernel<Tout><<<blocks, kGatherThreads, smem, stream>>>(src.Y, n, src.X, m, rows, kr, src.d, inv2s2, Rt));
    }
  }
  if (W && C && kr > 0 && kc > 0) {
    const int total = kr * kc;
    CABS_LAUNCH(stream, "w_from_c_kernel", w_from_c_kernel<Tout><<<ceil_div(total, 256), 256, 0, stream>>>(C, m, kc, rows, kr, W));
  }
  return CABS_OK;
}

}  // namespace

cabs_status launch_gather(const cabs_source& src, int64_t m, int64_t n, const int* rows, int kr, const int* cols,
                          int kc, bool elem_f64, void* C, void* Rt, double* W, cudaStream_t stream) {
  if (elem_f64)
    return gather_typed<double>(src, m, n, rows, kr, cols, kc, (double*)C, (double*)Rt, W, stream);
  return gather_typed<float>(src, m, n, rows, kr, cols, kc, (float*)C, (float*)Rt, W, stream);
}

cabs_status launch_rows_of(const void* C, int64_t m, int kc, const int* rows, int kr, bool elem_f64, double* W,
                           cudaStream_t stream) {
  const int total = kr * kc;
  if (total <= 0) return CABS_OK;
  if (elem_f64)
    CABS_LAUNCH(stream, "w_from_c_kernel",
                w_from_c_kernel<double><<<ceil_div(total, 256), 256, 0, stream>>>((const double*)C, m, kc, rows, kr, W));
  else
    CABS_LAUNCH(stream, "w_from_c_kernel",
                w_from_c_kernel<float><<<ceil_div(total, 256), 256, 0, stream>>>((const float*)C, m, kc, rows, kr, W));
  return CABS_OK;
}

}  // namespace cabs
