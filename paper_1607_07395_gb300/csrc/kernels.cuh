// Host-side launchers of the hot-path kernels (internal, not part of the ABI).
// Every launcher validates nothing beyond what its kernel needs, enqueues on
// `stream`, and returns CABS_ECUDA if the launch failed.
#pragma once

#include "common.cuh"

namespace cabs {

// a1: two independent draws (rows and columns) in one launch; pass k1 = 0 for one.
cabs_status launch_draw2(uint64_t seed, int tag0, long long N0, int k0, int* drawn0, int* sorted0, int tag1,
                         long long N1, int k1, int* drawn1, int* sorted1, cudaStream_t stream);

// a2/a7: gathers. `elem_f64` selects the output element type of C and Rt.
cabs_status launch_gather(const cabs_source& src, int64_t m, int64_t n, const int* rows, int kr, const int* cols,
                          int kc, bool elem_f64, void* C, void* Rt, double* W, cudaStream_t stream);

// a3/a4/a8: the sketching routine. Workspace bytes for (m, n, k, elem).
size_t core_ws_bytes(int64_t m, int64_t n, int k, bool elem_f64);
// tc_ok: an FP32 (not FP64) sketch in the BF16 or TF32 mode, whose
// extrapolation products may run on the tensor cores (3 x TF32, k <= 256).
cabs_status launch_core(int64_t m, int64_t n, int k, bool elem_f64, bool tc_ok, int core, double trunc_rtol,
                        const void* C, const void* Rt, const double* W, bool embed, void* out1, double* S, void* out2,
                        int* d_rank, int* d_sweeps, int* d_refine, int* d_status, double* d_sig, double* d_Uw,
                        double* d_Vw, void* ws, size_t ws_bytes, cudaStream_t stream);

// out (M x N, elem) = X (M x K, elem) * B (K x N, FP64), with the FP64 sum of
// squares of each output column over each block of rows in part
// (extrap_row_blocks(M) x N).
int extrap_row_blocks(int64_t M, bool elem_f64);
cabs_status launch_extrap_gemm(const void* X, int64_t M, int K, const double* B, int N, bool elem_f64, void* out,
                               double* part, const char* name, cudaStream_t stream);

// The two extrapolation products a = C V_w (m x k) and b = Rt U_w (n x k) on
// the tensor cores, 3 x TF32 (k <= 256); parts as launch_extrap_gemm with
// 128-row blocks; img: tc_extrap_img_bytes(k) of scratch; a wait that runs
// out sets bit value 4 of *status (may be NULL).
size_t tc_extrap_img_bytes(int k);
cabs_status launch_tc_extrap_pair(const float* C, int64_t m, const float* Rt, int64_t n, int k, const double* Vw,
                                  const double* Uw, float* out1, float* out2, double* part1, double* part2, void* img,
                                  int* status, cudaStream_t stream);

// G = X^T X (K x K, FP64) of a tall X (M x K, elem); part: gram_ws_bytes(M, K) of scratch.
size_t gram_ws_bytes(int64_t M, int K, bool elem_f64);
cabs_status launch_gram(const void* X, int64_t M, int K, bool elem_f64, void* part, double* G, cudaStream_t stream);

// k x k FP64 product C = diag(a) op(A) diag(d) op(B) diag(b) (a, b, d may be NULL).
cabs_status launch_kk_gemm(int k, const double* A, bool transA, const double* d, const double* B, bool transB,
                           const double* a, const double* b, double* C, cudaStream_t stream);

// FP64 C (M x N) = op(A) diag(d) op(B) for small row-major operands.
cabs_status launch_small_gemm(int M, int N, int K, const double* A, int lda, bool transA, const double* d,
                              const double* B, int ldb, bool transB, double* C, int ldc, cudaStream_t stream);

// Supplementary Section 3: U diag(S) V^T -> X diag(s) Y^T with orthonormal X, Y.
size_t orth_ws_bytes(int64_t m, int64_t n, int k, bool elem_f64);
cabs_status launch_orthogonalize(int64_t m, int64_t n, int k, bool elem_f64, double trunc_rtol, const void* U,
                                 const double* S, const void* V, void* X, double* s, void* Y, int* d_rank,
                                 int* d_status, void* ws, size_t ws_bytes, cudaStream_t stream);

// a5: weighted k-means.
size_t kmeans_ws_bytes(int64_t M, int d, int k2, int iters, int prec);
cabs_status launch_kmeans(const void* X, int64_t M, int d, const int* init_rows, int k2, int iters, int prec,
                          float upsilon_pow, int* labels, void* centres, double* energy, int* d_T, int* d_recheck,
                          void* ws, size_t ws_bytes, cudaStream_t stream);
// Weighted encoding error of X with representatives X[reps] (k2 rows), nearest assignment.
cabs_status launch_encoding_error(const void* X, int64_t M, int d, const int* reps, int k2, int prec,
                                  float upsilon_pow, double* out, void* ws, size_t ws_bytes, cudaStream_t stream);

// a6: snap.
size_t snap_ws_bytes(int64_t M, int d, int k2, int prec);
// status (may be NULL): bit 2 is set when a grid barrier of the walk gave up.
cabs_status launch_snap(const void* X, int64_t M, int d, const void* Z, int k2, int prec, int* order, int* sorted,
                        void* ws, size_t ws_bytes, int* fallbacks, int* status, cudaStream_t stream);

// Section 5 follow-up variant (f): the k2 largest-norm rows of X, sorted.
size_t threshold_ws_bytes(int64_t M);
cabs_status launch_threshold(const void* X, int64_t M, int d, int k2, int prec, int* sorted, void* ws,
                             size_t ws_bytes, cudaStream_t stream);
// Section 5 follow-up variant (e): k2 distinct rows drawn with probabilities
// proportional to the leverage scores |X_i|^2 of an orthonormal X (A-Res keys,
// Philox key (seed, tag)), sorted. Workspace: threshold_ws_bytes(M).
cabs_status launch_leverage_select(const void* X, int64_t M, int d, int k2, bool elem_f64, uint64_t seed, int tag,
                                   int* sorted, void* ws, size_t ws_bytes, cudaStream_t stream);

// W[p][t] = C[rows[p]][t] (kr x kc, FP64) from C (m x kc, elem).
cabs_status launch_rows_of(const void* C, int64_t m, int kc, const int* rows, int kr, bool elem_f64, double* W,
                           cudaStream_t stream);

// Section 2.2, Algorithm 1: Sketch-CUR.
size_t cur_ws_bytes(int64_t m, int64_t n, int kb, int kt, bool elem_f64);
cabs_status launch_sketch_cur(const cabs_source& src, int64_t m, int64_t n, int kb, int kt, uint64_t seed,
                              bool elem_f64, double trunc_rtol, void* U, double* S, void* V, double* Ustar,
                              int* rows_b, int* cols_b, int* rows_t, int* cols_t, int* ranks, void* ws,
                              size_t ws_bytes, cudaStream_t stream);

// a9: relative Frobenius error.
size_t error_ws_bytes(const cabs_source& src, int64_t m, int64_t n, int k, int64_t samples, int prec);
size_t tc_residual_ws_bytes(int64_t m, int64_t n, int k, bool tf32);
cabs_status launch_tc_residual(const cabs_source& src, int64_t m, int64_t n, int k, bool tf32, const float* U,
                               const double* S, const float* V, void* ws, size_t ws_bytes, double* out2,
                               cudaStream_t stream);
cabs_status launch_error(const cabs_source& src, int64_t m, int64_t n, int k, bool elem_f64, int prec,
                         const void* U, const double* S, const void* V, int64_t samples, uint64_t seed, void* ws,
                         size_t ws_bytes, double* d_out2 /* num, den */, cudaStream_t stream);

}  // namespace cabs
