// Sketch-CUR: Bilateral Resampling CUR (Section 2.2, Algorithm 1) with
// independent uniform base and target samplings (Section 2.2, item 3; the
// comparison (a) of Section 5 samples the target at three times the base).
//
//  1. Draws: base rows / columns (k_b each, the pilot draw of Algorithm 2,
//     tags 0 and 1) and target rows / columns (k_t each, tags 4 and 5).
//  2. Bases: C = A[:, I^b_c] (m x k_b, elem) and R^T = A[I^b_r, :]^T
//     (n x k_b, elem, straight into the output V).
//  3. Targets: the target columns A[:, I^t_c] (m x k_t, elem, scratch) give
//     M = A[I^t_r, I^t_c] and R_bar = A[I^b_r, I^t_c]; C gives
//     C_bar = A[I^t_r, I^b_c]; all three in FP64.
//  4. U* = C_bar^+ M R_bar^+ in FP64 (step 4). Each pseudo-inverse comes
//     from the FP64-accurate SVD of the sketching routine applied to the
//     tall orientation of the block (B, or B^T when B is wide) padded with
//     zero columns to K x K (K = max(k_b, k_t)): the SVD's refinement takes
//     the kept columns of U from W V in FP64, so zero columns cost nothing
//     in accuracy. Kept: sigma_i > max(trunc_rtol, K 2^-52) sigma_1 (MATLAB
//     pinv's default floor, as in the sketching routine; data carried in
//     FP32 pass their resolution K 2^-24 in trunc_rtol).
//     pinv(pad) = V Sigma^+ U^T holds B^+ (or (B^+)^T) in its first rows.
//  5. A ~ C U* R returned as U = C U* (m x k_b, CUDA cores), S = 1, V = R^T.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "svd.cuh"

namespace cabs {
namespace {

constexpr int kTagTargetRows = 4;
constexpr int kTagTargetCols = 5;

// out (K x K): the tall orientation of in (r x c, row-major) -- in itself
// when r >= c, in^T otherwise -- in the top-left corner, zero elsewhere.
__global__ void pad_tall_kernel(const double* __restrict__ in, int r, int c, int K, double* __restrict__ out) {
  const bool tr = r < c;
  const int rr = tr ? c : r, cc = tr ? r : c;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x) {
    const int i = e / K, j = e - i * K;
    double v = 0.0;
    if (i < rr && j < cc) v = tr ? in[(size_t)j * c + i] : in[(size_t)i * c + j];
    out[e] = v;
  }
}

// inv[i] = 1 / sig[i] for i < rank (and sig[i] > 0), else 0.
__global__ void recip_kernel(int n, const double* __restrict__ sig, const int* __restrict__ rank,
                             double* __restrict__ inv) {
  const int r = *rank;
  for (int i = threadIdx.x; i < n; i += blockDim.x) inv[i] = (i < r && sig[i] > 0.0) ? 1.0 / sig[i] : 0.0;
}

// out (rows x cols) = P[0:rows, 0:cols] or, with tr, P[0:cols, 0:rows]^T (P: K x K).
__global__ void take_block_kernel(const double* __restrict__ P, int K, int rows, int cols, int tr,
                                  double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < rows * cols; e += gridDim.x * blockDim.x) {
    const int i = e / cols, j = e - i * cols;
    out[e] = tr ? P[(size_t)j * K + i] : P[(size_t)i * K + j];
  }
}

// S = 1 (the factor form of C U* R).
__global__ void ones_kernel(int kb, double* __restrict__ S) {
  for (int i = threadIdx.x; i < kb; i += blockDim.x) S[i] = 1.0;
}

struct CurWs {
  SvdWs svd;
  int *rb_drawn, *cb_drawn, *rt_drawn, *ct_drawn;
  void *C, *Ct;
  double *Cbar, *Rbar, *M, *Pad, *Usv, *Vsv, *Pinv, *sig, *isig, *Cp, *Rp, *T, *Ustar;
  double* part;
  int* ranks;
};

CurWs carve_cur(Carve& cv, int64_t m, int64_t n, int kb, int kt, bool f64) {
  CurWs w;
  const int K = std::max(kb, kt);
  const size_t eb = f64 ? 8 : 4, KK = (size_t)K * K, BT = (size_t)kb * kt;
  w.svd = carve_svd(cv, K);
  w.rb_drawn = cv.take<int>(kb);
  w.cb_drawn = cv.take<int>(kb);
  w.rt_drawn = cv.take<int>(kt);
  w.ct_drawn = cv.take<int>(kt);
  w.C = cv.take<char>((size_t)m * kb * eb);
  w.Ct = cv.take<char>((size_t)m * kt * eb);
  w.Cbar = cv.take<double>(BT);
  w.Rbar = cv.take<double>(BT);
  w.M = cv.take<double>((size_t)kt * kt);
  double** sq[] = {&w.Pad, &w.Usv, &w.Vsv, &w.Pinv};
  for (double** p : sq) *p = cv.take<double>(KK);
  w.sig = cv.take<double>(K);
  w.isig = cv.take<double>(K);
  w.Cp = cv.take<double>(BT);
  w.Rp = cv.take<double>(BT);
  w.T = cv.take<double>(BT);
  w.Ustar = cv.take<double>((size_t)kb * kb);
  w.part = cv.take<double>((size_t)extrap_row_blocks(m, f64) * kb);
  w.ranks = cv.take<int>(8);
  return w;
}

// B^+ (c x r) of B (r x c) into out; diagnostics into rk[which], rk[2 + which], ...
cabs_status pinv_block(const CurWs& w, const double* B, int r, int c, int K, double tol, double res, double* out,
                       int* rk, int which, cudaStream_t stream) {
  const int pb = std::max(1, std::min(ceil_div(K * K, 256), 4 * sm_count()));
  CABS_LAUNCH(stream, "pad_tall_kernel", pad_tall_kernel<<<pb, 256, 0, stream>>>(B, r, c, K, w.Pad));
  CABS_TRY(launch_svd(w.Pad, K, tol, res, w.sig, w.Usv, w.Vsv, &rk[which], &rk[2 + which], &rk[4 + which], &rk[6],
                      w.svd, stream));
  CABS_LAUNCH(stream, "recip_kernel", recip_kernel<<<1, 256, 0, stream>>>(K, w.sig, &rk[which], w.isig));
  CABS_TRY(launch_kk_gemm(K, w.Vsv, false, w.isig, w.Usv, true, nullptr, nullptr, w.Pinv, stream));
  // tall B: B^+ = Pinv[0:c, 0:r]; wide B: Pinv[0:r, 0:c] = (B^+)^T
  const int tb = std::max(1, std::min(ceil_div(r * c, 256), 4 * sm_count()));
  CABS_LAUNCH(stream, "take_block_kernel",
              take_block_kernel<<<tb, 256, 0, stream>>>(w.Pinv, K, c, r, r < c ? 1 : 0, out));
  return CABS_OK;
}

}  // namespace

size_t cur_ws_bytes(int64_t m, int64_t n, int kb, int kt, bool elem_f64) {
  Carve cv;
  carve_cur(cv, m, n, kb, kt, elem_f64);
  return cv.used;
}

cabs_status launch_sketch_cur(const cabs_source& src, int64_t m, int64_t n, int kb, int kt, uint64_t seed,
                              bool f64, double trunc_rtol, void* U, double* S, void* V, double* Ustar_out,
                              int* rows_b, int* cols_b, int* rows_t, int* cols_t, int* ranks, void* ws,
                              size_t ws_bytes, cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  CurWs w = carve_cur(cv, m, n, kb, kt, f64);
  if (!cv.fits()) {
    set_error("Sketch-CUR workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  const int K = std::max(kb, kt);
  int* rk = ranks ? ranks : w.ranks;
  if (cudaMemsetAsync(rk, 0, 8 * sizeof(int), stream) != cudaSuccess) return check_cuda("cur diagnostics clear");
  // 1. base and target draws
  CABS_TRY(launch_draw2(seed, 0, m, kb, w.rb_drawn, rows_b, 1, n, kb, w.cb_drawn, cols_b, stream));
  CABS_TRY(launch_draw2(seed, kTagTargetRows, m, kt, w.rt_drawn, rows_t, kTagTargetCols, n, kt, w.ct_drawn, cols_t,
                        stream));
  // 2. bases C and R^T
  CABS_TRY(launch_gather(src, m, n, rows_b, kb, cols_b, kb, f64, w.C, V, nullptr, stream));
  // 3. target columns -> M, R_bar; C -> C_bar
  CABS_TRY(launch_gather(src, m, n, rows_t, kt, cols_t, kt, f64, w.Ct, nullptr, w.M, stream));
  CABS_TRY(launch_rows_of(w.Ct, m, kt, rows_b, kb, f64, w.Rbar, stream));  // kb x kt
  CABS_TRY(launch_rows_of(w.C, m, kb, rows_t, kt, f64, w.Cbar, stream));   // kt x kb
  // 4. pseudo-inverses and U* = (C_bar^+ M) R_bar^+
  const double tol = std::max(trunc_rtol, (double)K * 2.220446049250313e-16);
  const double res = f64 ? 0.0 : kResolveReduced;
  CABS_TRY(pinv_block(w, w.Cbar, kt, kb, K, tol, res, w.Cp, rk, 0, stream));  // kb x kt
  CABS_TRY(pinv_block(w, w.Rbar, kb, kt, K, tol, res, w.Rp, rk, 1, stream));  // kt x kb
  CABS_TRY(launch_small_gemm(kb, kt, kt, w.Cp, kt, false, nullptr, w.M, kt, false, w.T, kt, stream));
  double* Us = Ustar_out ? Ustar_out : w.Ustar;
  CABS_TRY(launch_small_gemm(kb, kb, kt, w.T, kt, false, nullptr, w.Rp, kb, false, Us, kb, stream));
  CABS_LAUNCH(stream, "ones_kernel", ones_kernel<<<1, 256, 0, stream>>>(kb, S));
  // 5. U = C U*
  return launch_extrap_gemm(w.C, m, kb, Us, kb, f64, U, w.part, "extrap_gemm_kernel(C U*)", stream);
}

}  // namespace cabs
