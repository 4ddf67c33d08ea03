// Steps a3 / a4 / a8 -- the sketching routine of Section 4.1 and the pilot
// embedding of Algorithm 2, step 2.
//
//  1. SVD W = U_w Sigma_w V_w^T to FP64 accuracy (svd.cu: FP32 one-sided
//     Jacobi on a thread-block cluster, then an FP64 refinement spread over
//     the GPU).
//  2. Truncation: keep sigma_i > max(trunc_rtol, k 2^-52) sigma_1; dropped
//     components get zero columns in U_w and V_w, hence zero factors and S.
//  3. Extrapolation a = C V_w (m x k), b = Rt U_w (n x k): on CUDA cores in
//     the working precision (FP64, FP32 modes), or on the tensor cores as
//     three TF32 products to FP32-level accuracy in the BF16 and TF32 modes
//     (tc_extrap.cu, k <= 256); each CTA also writes the FP64 sum of squares
//     of its 128-row tile's columns, and the norms N_c, N_r are reduced by
//     one CTA per column in a fixed order (deterministic).
//  4. Scale: S_i = N_c,i N_r,i / sigma_i (pseudo-skeleton C W^+ R, Eq. W) or
//     S_i = sigma_i sqrt(mn)/k (stabilised form); the factors are
//     U = a N_c^-1, V = b N_r^-1, or the embeddings P = U S^1/2, Q = V S^1/2.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "svd.cuh"

namespace cabs {
namespace {

// out[M x N] = X[M x K] * B[K x N] with X in T and B in FP64 (converted to T);
// N = K = k. Also the FP64 sum of squares of each output column over this
// CTA's rows: part[blockIdx.y * N + col]. 256 threads; each thread owns a
// TM x TN register tile (8 x 8 in FP32, 4 x 4 in FP64), so one CTA covers
// (16 TM) x (16 TN) outputs and reads 2 (TM + TN) / 4 shared-memory vectors
// per TM TN multiply-adds. Every output sums over K in ascending order, as a
// plain loop would, whatever the tile shape.
constexpr int kGBK = 16;
// The output columns per thread (TN) are a launch shape: the row tiling (TM,
// BM) fixes the per-CTA column partials, so any TN gives identical results.
template <typename T>
struct ExtrapTile {
  static constexpr int TM = sizeof(T) == 4 ? 8 : 4;
  static constexpr int TN = sizeof(T) == 4 ? 8 : 4;
  static constexpr int BM = 16 * TM, BN = 16 * TN;
};

template <typename T, int TN = ExtrapTile<T>::TN>
__global__ void __launch_bounds__(256) extrap_gemm_kernel(const T* __restrict__ X, long long M, int K,
                                                         const double* __restrict__ B, int N, T* __restrict__ out,
                                                         double* __restrict__ part) {
  constexpr int TM = ExtrapTile<T>::TM;
  constexpr int BM = ExtrapTile<T>::BM, BN = 16 * TN;
  constexpr int LA = BM * kGBK / 256, LB = BN * kGBK / 256;  // elements each thread stages per chunk
  // A and B double buffers; the column sums reuse the space after the loop
  constexpr size_t kAB = sizeof(T) * 2 * kGBK * ((BM + 4) + (BN + 4));
  constexpr size_t kCS = sizeof(double) * 16 * BN;
  __shared__ __align__(16) unsigned char ext_smem[kAB > kCS ? kAB : kCS];
  auto As = reinterpret_cast<T(*)[kGBK][BM + 4]>(ext_smem);
  auto Bs = reinterpret_cast<T(*)[kGBK][BN + 4]>(ext_smem + sizeof(T) * 2 * kGBK * (BM + 4));
  auto colsq = reinterpret_cast<double(*)[BN]>(ext_smem);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long m0 = (long long)blockIdx.y * BM;
  const int n0 = blockIdx.x * BN;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  // the next chunk is read from global memory into registers while the
  // current one is multiplied out of shared memory (two shared buffers)
  T ra[LA], rb[LB];
  auto load = [&](int k0) {
#pragma unroll
    for (int e = 0; e < LA; ++e) {
      const int idx = tid + 256 * e;
      const int r = idx >> 4, c = idx & 15;  // X tile: BM rows x 16 k, read along k
      const long long gm = m0 + r;
      const int gk = k0 + c;
      ra[e] = (gm < M && gk < K) ? X[gm * K + gk] : T(0);
    }
#pragma unroll
    for (int e = 0; e < LB; ++e) {
      const int idx = tid + 256 * e;
      const int br = idx / BN, bc = idx - br * BN;  // B tile: 16 k x BN cols
      const int bk = k0 + br, bn = n0 + bc;
      rb[e] = (bk < K && bn < N) ? (T)B[(size_t)bk * N + bn] : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < LA; ++e) {
      const int idx = tid + 256 * e;
      As[buf][idx & 15][idx >> 4] = ra[e];
    }
#pragma unroll
    for (int e = 0; e < LB; ++e) {
      const int idx = tid + 256 * e;
      const int br = idx / BN;
      Bs[buf][br][idx - br * BN] = rb[e];
    }
  };
  load(0);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = 0; k0 < K; k0 += kGBK) {
    const bool more = k0 + kGBK < K;
    if (more) load(k0 + kGBK);
#pragma unroll
    for (int kk = 0; kk < kGBK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[buf][kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[buf][kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  T sq[TN];
#pragma unroll
  for (int j = 0; j < TN; ++j) sq[j] = T(0);
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const long long gm = m0 + ty * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx * TN + j;
      if (gn < N) {
        out[gm * N + gn] = acc[i][j];
        sq[j] = fma(acc[i][j], acc[i][j], sq[j]);
      }
    }
  }
#pragma unroll
  for (int j = 0; j < TN; ++j) colsq[ty][tx * TN + j] = (double)sq[j];
  __syncthreads();
  if (tid < BN) {
    double s2 = 0.0;
    for (int r = 0; r < 16; ++r) s2 += colsq[r][tid];
    const int gn = n0 + tid;
    if (gn < N) part[(size_t)blockIdx.y * N + gn] = s2;
  }
}

// One CTA per column r: its norms N_c, N_r from the per-row-block partials
// (summed by a fixed tree over the CTA's threads, so deterministic), then S
// and the column's two scale factors.
__global__ void __launch_bounds__(256) core_finalize_kernel(const double* __restrict__ part1, int nb1,
                                                            const double* __restrict__ part2, int nb2, int k,
                                                            const double* __restrict__ sig,
                                                            const int* __restrict__ rank_p, int core, int embed,
                                                            double mn_over_kk, double* __restrict__ S,
                                                            double* __restrict__ f1, double* __restrict__ f2) {
  __shared__ double red[2][256];
  const int r = blockIdx.x, tid = threadIdx.x;
  double s1 = 0.0, s2 = 0.0;
  for (int b = tid; b < nb1; b += blockDim.x) s1 += part1[(size_t)b * k + r];
  for (int b = tid; b < nb2; b += blockDim.x) s2 += part2[(size_t)b * k + r];
  red[0][tid] = s1;
  red[1][tid] = s2;
  __syncthreads();
  for (int w = blockDim.x >> 1; w > 0; w >>= 1) {
    if (tid < w) {
      red[0][tid] += red[0][tid + w];
      red[1][tid] += red[1][tid + w];
    }
    __syncthreads();
  }
  if (tid != 0) return;
  const double nc = sqrt(red[0][0]), nr = sqrt(red[1][0]);
  const int rank = *rank_p;
  double sv = 0.0, a = 0.0, c = 0.0;
  if (r < rank && nc > 0.0 && nr > 0.0) {
    sv = (core == CABS_CORE_STABILIZED) ? sig[r] * sqrt(mn_over_kk) : nc * nr / sig[r];
    const double e = embed ? sqrt(sv) : 1.0;
    a = e / nc;
    c = e / nr;
  }
  S[r] = sv;
  f1[r] = a;
  f2[r] = c;
}

template <typename T>
__global__ void scale_cols_kernel(T* __restrict__ X, long long M, int k, const double* __restrict__ f) {
  __shared__ T fs[CABS_MAX_K];
  for (int r = threadIdx.x; r < k; r += blockDim.x) fs[r] = (T)f[r];
  __syncthreads();
  const long long total = M * k;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e % k);
    X[e] *= fs[r];
  }
}

struct CoreWs {
  SvdWs svd;
  double *sig, *Uw, *Vw, *part1, *part2, *f1, *f2;
  int *rank, *sweeps;
  void* img;  // tensor-core extrapolation: B images
};

CoreWs carve_core(Carve& cv, int64_t m, int64_t n, int k) {
  CoreWs w;
  w.svd = carve_svd(cv, k);
  w.sig = cv.take<double>(k);
  w.Uw = cv.take<double>((size_t)k * k);
  w.Vw = cv.take<double>((size_t)k * k);
  // column-norm partials: one row per CTA row block (the FP64 tile is the shorter)
  w.part1 = cv.take<double>((size_t)ceil_div(m, ExtrapTile<double>::BM) * k);
  w.part2 = cv.take<double>((size_t)ceil_div(n, ExtrapTile<double>::BM) * k);
  w.f1 = cv.take<double>(k);
  w.f2 = cv.take<double>(k);
  w.rank = cv.take<int>(1);
  w.sweeps = cv.take<int>(1);
  w.img = k <= 256 ? (void*)cv.take<char>(tc_extrap_img_bytes(k)) : nullptr;
  return w;
}

// The two extrapolation products C V_w and R^T U_w with TN output columns
// per thread (the launch shape of the sketch's bucket; 0 = the default).
template <typename T, int TN>
cabs_status extrap_pair_tn(const T* C, int64_t m, const T* Rt, int64_t n, int k, const double* Vw, const double* Uw,
                           T* out1, T* out2, double* part1, double* part2, cudaStream_t stream) {
  constexpr int BM = ExtrapTile<T>::BM, BN = 16 * TN;
  dim3 g1(ceil_div(k, BN), ceil_div(m, BM)), g2(ceil_div(k, BN), ceil_div(n, BM));
  CABS_LAUNCH(stream, "extrap_gemm_kernel(C V_w)",
              (extrap_gemm_kernel<T, TN><<<g1, 256, 0, stream>>>(C, m, k, Vw, k, out1, part1)));
  CABS_LAUNCH(stream, "extrap_gemm_kernel(Rt U_w)",
              (extrap_gemm_kernel<T, TN><<<g2, 256, 0, stream>>>(Rt, n, k, Uw, k, out2, part2)));
  return CABS_OK;
}

template <typename T>
cabs_status extrap_pair(int tn, const T* C, int64_t m, const T* Rt, int64_t n, int k, const double* Vw,
                        const double* Uw, T* out1, T* out2, double* part1, double* part2, cudaStream_t stream) {
  if (tn == 2) return extrap_pair_tn<T, 2>(C, m, Rt, n, k, Vw, Uw, out1, out2, part1, part2, stream);
  if (tn == 4) return extrap_pair_tn<T, 4>(C, m, Rt, n, k, Vw, Uw, out1, out2, part1, part2, stream);
  if constexpr (sizeof(T) == 4)
    if (tn == 8) return extrap_pair_tn<T, 8>(C, m, Rt, n, k, Vw, Uw, out1, out2, part1, part2, stream);
  return extrap_pair_tn<T, ExtrapTile<T>::TN>(C, m, Rt, n, k, Vw, Uw, out1, out2, part1, part2, stream);
}

template <typename T>
cabs_status core_typed(int64_t m, int64_t n, int k, bool tc_ok, int core, double trunc_rtol, const T* C, const T* Rt,
                       const double* W, bool embed, T* out1, double* S, T* out2, int* d_rank, int* d_sweeps,
                       int* d_refine, int* d_status, double* d_sig, double* d_Uw, double* d_Vw, void* ws, size_t ws_bytes,
                       cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  CoreWs w = carve_core(cv, m, n, k);
  if (!cv.fits()) {
    set_error("core workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  double* sig = d_sig ? d_sig : w.sig;
  double* Uw = d_Uw ? d_Uw : w.Uw;
  double* Vw = d_Vw ? d_Vw : w.Vw;
  int* rank = d_rank ? d_rank : w.rank;
  int* sweeps = d_sweeps ? d_sweeps : w.sweeps;
  CABS_TRY(launch_svd(W, k, trunc_rtol, sizeof(T) == 8 ? 0.0 : kResolveReduced, sig, Uw, Vw, rank, sweeps, d_refine,
                      d_status, w.svd, stream));
  const int nb1 = ceil_div(m, ExtrapTile<T>::BM), nb2 = ceil_div(n, ExtrapTile<T>::BM);
  bool done = false;
  if constexpr (sizeof(T) == 4) {
    if (tc_ok && k <= 256) {
      // 128-row blocks, as the FP32 CUDA-core tile (nb1, nb2 above)
      CABS_TRY(launch_tc_extrap_pair(C, m, Rt, n, k, Vw, Uw, out1, out2, w.part1, w.part2, w.img, d_status, stream));
      done = true;
    }
  }
  if (!done) {
    const int tn = current_tune().extrap_tn;
    CABS_TRY(extrap_pair<T>(tn, C, m, Rt, n, k, Vw, Uw, out1, out2, w.part1, w.part2, stream));
  }
  const double mn_over_kk = (double)m * (double)n / ((double)k * (double)k);
  CABS_LAUNCH(stream, "core_finalize_kernel",
              core_finalize_kernel<<<k, 256, 0, stream>>>(w.part1, nb1, w.part2, nb2, k, sig, rank, core, embed ? 1 : 0,
                                                          mn_over_kk, S, w.f1, w.f2));
  const int sms = sm_count();
  CABS_LAUNCH(stream, "scale_cols_kernel(1)", scale_cols_kernel<T><<<std::max(1, std::min(ceil_div(m * k, 256), sms * 8)), 256, 0, stream>>>(out1, m, k, w.f1));
  CABS_LAUNCH(stream, "scale_cols_kernel(2)", scale_cols_kernel<T><<<std::max(1, std::min(ceil_div(n * k, 256), sms * 8)), 256, 0, stream>>>(out2, n, k, w.f2));
  return CABS_OK;
}

}  // namespace

int extrap_row_blocks(int64_t M, bool elem_f64) {
  return ceil_div(M, elem_f64 ? ExtrapTile<double>::BM : ExtrapTile<float>::BM);
}

cabs_status launch_extrap_gemm(const void* X, int64_t M, int K, const double* B, int N, bool elem_f64, void* out,
                               double* part, const char* name, cudaStream_t stream) {
  if (elem_f64) {
    dim3 g(ceil_div(N, ExtrapTile<double>::BN), ceil_div(M, ExtrapTile<double>::BM));
    CABS_LAUNCH(stream, name,
                extrap_gemm_kernel<double><<<g, 256, 0, stream>>>((const double*)X, M, K, B, N, (double*)out, part));
  } else {
    dim3 g(ceil_div(N, ExtrapTile<float>::BN), ceil_div(M, ExtrapTile<float>::BM));
    CABS_LAUNCH(stream, name,
                extrap_gemm_kernel<float><<<g, 256, 0, stream>>>((const float*)X, M, K, B, N, (float*)out, part));
  }
  return CABS_OK;
}

size_t core_ws_bytes(int64_t m, int64_t n, int k, bool /*elem_f64*/) {
  Carve cv;
  carve_core(cv, m, n, k);
  return cv.used;
}

cabs_status launch_core(int64_t m, int64_t n, int k, bool elem_f64, bool tc_ok, int core, double trunc_rtol,
                        const void* C, const void* Rt, const double* W, bool embed, void* out1, double* S, void* out2,
                        int* d_rank, int* d_sweeps, int* d_refine, int* d_status, double* d_sig, double* d_Uw,
                        double* d_Vw, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (elem_f64)
    return core_typed<double>(m, n, k, false, core, trunc_rtol, (const double*)C, (const double*)Rt, W, embed,
                              (double*)out1, S, (double*)out2, d_rank, d_sweeps, d_refine, d_status, d_sig, d_Uw, d_Vw, ws,
                              ws_bytes, stream);
  return core_typed<float>(m, n, k, tc_ok, core, trunc_rtol, (const float*)C, (const float*)Rt, W, embed, (float*)out1, S,
                           (float*)out2, d_rank, d_sweeps, d_refine, d_status, d_sig, d_Uw, d_Vw, ws, ws_bytes, stream);
}

}  // namespace cabs
