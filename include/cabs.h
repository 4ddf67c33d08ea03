/*
 * cabs.h -- C ABI of libcabs, a single-GPU (GB300, sm_103a) implementation of
 * cascaded bilateral sampling (CABS; Zhang, Liu, Zhang, Xiong, Xing, Ye,
 * "Seeing the Forest from the Trees in Two Looks: Matrix Sketching by Cascaded
 * Bilateral Sampling", arXiv 1607.07395).
 *
 * Problem (Algorithm 2): given an m x n matrix A that is read only through a
 * few of its rows and columns, return A ~ U_bar diag(S_bar) V_bar^T and the
 * sampled row and column indices.
 *
 * Conventions for every call below
 *  - Pointers named d_* or documented as "device" are CUDA device pointers of
 *    the current device; "host" pointers are ordinary CPU memory.
 *  - Matrices are row-major. A is m x n with leading dimension lda >= n.
 *    C (m x k) holds the sampled columns A[:, J]; R is kept transposed,
 *    Rt (n x k) = A[I, :]^T, as in the proof of Theorem 1 of the paper.
 *  - The working element type ("elem") is double when prec == CABS_PREC_FP64
 *    and float otherwise. W, Sigma_w, S and every k x k core quantity are
 *    always double (the core solve stays in FP64).
 *  - Index arrays are int32 and 0-based.
 *  - Work is enqueued on the given CUDA stream (a cudaStream_t passed as
 *    void*; NULL = the legacy default stream) and the call returns without
 *    waiting, unless its comment says otherwise. Outputs are valid once the
 *    stream reaches that point.
 *  - The caller owns every buffer it passes in, including workspaces; the
 *    library never frees or keeps them after the call returns (the serving
 *    loop keeps its arena until cabs_serve_stop). Inputs are never written.
 *  - Errors are reported by the returned status only; nothing aborts and no
 *    C++ exception crosses this interface. A readable message for the
 *    calling thread's last failure is available from cabs_last_error().
 *  - There is no CPU fallback: without a usable CUDA device every call that
 *    computes returns CABS_ECUDA.
 */
#ifndef CABS_H
#define CABS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#pragma GCC visibility push(default)
#endif

typedef struct cabs_ctx cabs_ctx;
typedef void* cabs_stream; /* cudaStream_t */

typedef enum {
  CABS_OK = 0,
  CABS_EINVAL = 1,   /* invalid argument (null pointer, size out of range, k > min(m, n), ...) */
  CABS_ENOMEM = 2,   /* a workspace or arena is smaller than required */
  CABS_ECUDA = 3,    /* a CUDA call or kernel launch failed */
  CABS_ETIMEOUT = 4, /* a bounded device-side wait gave up, or a host wait timed out */
  CABS_EBUSY = 5,    /* serving: no free slot / request still running */
  CABS_ERANK = 6,    /* W is numerically zero: no component survives truncation */
  CABS_ENOTFOUND = 7 /* serving: unknown ticket */
} cabs_status;

typedef enum {
  CABS_PREC_FP64 = 0, /* every step in FP64 (parity mode) */
  CABS_PREC_FP32 = 1, /* FP32 gathers, extrapolation, clustering; FP64 core */
  CABS_PREC_TF32 = 2, /* as FP32, k-means distance contraction on TF32 tensor cores */
  CABS_PREC_BF16 = 3  /* as FP32, k-means distance contraction on BF16 tensor cores */
} cabs_prec;

typedef enum {
  /* Pseudo-skeleton A ~ C W^+ R (Section 2.2, Eq. W): S_i = N_c,i N_r,i / sigma_i. */
  CABS_CORE_PINV = 0,
  /* Stabilised sketching routine (Section 4.1): S_i = sigma_i sqrt(m n) / k. */
  CABS_CORE_STABILIZED = 1
} cabs_core;

typedef enum { CABS_SRC_DENSE = 0, CABS_SRC_RBF = 1, CABS_SRC_CSR = 2 } cabs_source_kind;

/* Where the entries of A come from. */
typedef struct {
  int32_t kind;     /* cabs_source_kind */
  /* CABS_SRC_DENSE: A, device, row-major m x n, leading dimension lda >= n,
   * FP64 when a_is_f64 != 0, else FP32. */
  const void* A;
  int64_t lda;
  int32_t a_is_f64;
  /* CABS_SRC_RBF: A[i, j] = exp(-|x_i - y_j|^2 / (2 sigma^2)), generated on
   * demand in the working precision and never stored. X (m x d) and Y (n x d)
   * are device FP32 row-major; 1 <= d <= CABS_MAX_D; sigma > 0. */
  const float* X;
  const float* Y;
  int32_t d;
  float sigma;
  /* CABS_SRC_CSR: a sparse A (the sparse inputs of Table 1) in compressed
   * rows, device: row_ptr (m + 1, int64, row_ptr[0] = 0, non-decreasing,
   * row_ptr[m] = nnz), col_idx (nnz, int32, strictly increasing within each
   * row, in [0, n)) and the values in A (nnz, FP64 when a_is_f64 != 0, else
   * FP32); lda is unused. Entries not stored are zero. The kernels clamp
   * row_ptr to [0, nnz] and skip column indices outside [0, n), so malformed
   * arrays give wrong values but no out-of-bounds access; unsorted rows give
   * wrong values. */
  const int64_t* row_ptr;
  const int32_t* col_idx;
  int64_t nnz;
} cabs_source;

#define CABS_MAX_K 256      /* largest k1 / k2 the sketch accepts */
#define CABS_MAX_D 64       /* largest point dimension of the RBF generator */
#define CABS_MAX_ITERS 64   /* largest number of k-means iterations */

/* Parameters of one sketch (Algorithm 2). */
typedef struct {
  int64_t m, n;       /* A is m x n */
  int32_t k1;         /* pilot samples per side, 1 <= k1 <= min(m, n, CABS_MAX_K) */
  int32_t k2;         /* follow-up samples per side, 1 <= k2 <= k1 */
  int32_t iters;      /* k-means iterations c (Section 4: c = 5), 0..CABS_MAX_ITERS */
  uint64_t seed;      /* Philox key word 0 of the pilot draw */
  int32_t prec;       /* cabs_prec */
  int32_t core;       /* cabs_core */
  float upsilon_pow;  /* Upsilon(t) = t^p of Eq. wkmeans; 0 = unweighted */
  double trunc_rtol;  /* keep sigma_i > max(trunc_rtol, k 2^-52) sigma_1 */
  int32_t flags;      /* CABS_FLAG_* */
  /* With CABS_FLAG_ERROR: the relative error of the sketch (as cabs_error,
   * Section 5) over err_samples sampled entries drawn with key (err_seed, 2),
   * or exactly over every entry when err_samples == 0 (dense sources only). */
  int64_t err_samples;
  uint64_t err_seed;
} cabs_params;

#define CABS_FLAG_FOLLOW_ERR 1 /* also compute the follow-up encoding errors e_f */
#define CABS_FLAG_ERROR 2      /* also compute the relative error into cabs_result.err */
/* Follow-up rows and columns by hard threshold (Section 5, follow-up variant
 * (f)): the k2 rows of P and of Q with the largest norm (the argument of the
 * monotone weight), ties to the lower index, instead of the weighted k-means
 * and the snap. iters and upsilon_pow are then unused, and the k-means
 * diagnostics (e_rows, e_cols, T_rows, T_cols) stay zero. */
#define CABS_FLAG_HARD_THRESHOLD 4
/* Return the sketch in SVD form (supplementary Section 3, as
 * cabs_orthogonalize): U and V with orthonormal columns and S the singular
 * values of U diag(S) V^T in descending order; diag.rank_final is then the
 * rank that form keeps. */
#define CABS_FLAG_SVD_FORM 8
/* Follow-up rows and columns by leverage scores (Section 5, follow-up
 * variant (e)): the pilot sketch P Q^T is put in SVD form X diag(s) Y^T
 * (supplementary Section 3, as cabs_orthogonalize with S = 1), and k2 distinct
 * rows (columns) are drawn without replacement with probabilities
 * proportional to the leverage scores |X_i|^2 (|Y_j|^2): the k2 largest A-Res
 * keys u_i^(1/l_i) (Efraimidis and Spirakis, 2006), ranked as l_i / (-ln u_i)
 * in FP64, u_i = ((r_i >> 11) + 1/2) 2^-53, r_i = word 0 of
 * Philox((i, 0, 0, 0), (seed, 6)) for rows and (seed, 7) for columns, ties to
 * the lower index. Excludes CABS_FLAG_HARD_THRESHOLD; the k-means
 * diagnostics stay zero. */
#define CABS_FLAG_LEVERAGE 16

/* Device-side diagnostics, written by the kernels of one sketch. */
typedef struct {
  int32_t rank_pilot, rank_final;         /* kept singular values of W and W_bar */
  int32_t sweeps_pilot, sweeps_final;     /* FP32 Jacobi sweeps of the two SVDs of W */
  int32_t T_rows, T_cols;                 /* max cluster size (Eq. T) of the last assignment */
  int32_t status;                         /* bit 0: the FP64 Jacobi hit its sweep limit; bit 1: the
                                           * FP64 refinement did not converge and the FP64 Jacobi ran;
                                           * bit 2: a bounded device-side wait gave up */
  int32_t rechecked;                      /* reduced precision: assignments re-checked in FP32 */
  double e_rows[CABS_MAX_ITERS];          /* weighted encoding error per k-means iteration */
  double e_cols[CABS_MAX_ITERS];          /*   (iteration 0 = the pilot representatives) */
  double e_follow_rows, e_follow_cols;    /* with the snapped follow-up representatives */
  int32_t snap_fallbacks;                 /* centres whose 8 nearest rows were all taken */
  int32_t refine_pilot, refine_final;     /* FP64 refinement iterations of the two SVDs
                                           * (-1: the FP64 Jacobi fallback ran) */
  int32_t reserved;
} cabs_diag;

/* Where one sketch's outputs go. All device memory, allocated by the caller. */
typedef struct {
  void* U;              /* elem, m x k2 (ld k2): U_bar; columns >= rank are zero */
  double* S;            /* k2: S_bar (zeros beyond rank) */
  void* V;              /* elem, n x k2 (ld k2): V_bar */
  int32_t* rows;        /* k2: follow-up row indices I_bar^r, ascending */
  int32_t* cols;        /* k2: follow-up column indices I_bar^c, ascending */
  int32_t* pilot_rows;  /* k1: pilot row indices I^r, ascending */
  int32_t* pilot_cols;  /* k1: pilot column indices I^c, ascending */
  cabs_diag* diag;      /* optional (may be NULL) */
  double* err;          /* 1 double; required with CABS_FLAG_ERROR, else unused (may be NULL) */
} cabs_result;

/* ---------------------------------------------------------------- context */

/* Creates a context bound to CUDA device `device`. Returns CABS_ECUDA when the
 * device cannot be used, CABS_EINVAL when out is NULL. */
cabs_status cabs_create(cabs_ctx** out, int device);
/* Destroys a context (stops its serving loop if one runs). NULL is a no-op. */
void cabs_destroy(cabs_ctx* ctx);
/* Message for the calling thread's last failure ("" if none). Never NULL. */
const char* cabs_last_error(cabs_ctx* ctx);
/* Library version string. */
const char* cabs_version(void);

/* Polls a grid-wide barrier of a cooperative kernel (the FP64 refinement of
 * the core SVD, the snap's greedy walk) makes before it gives up; a barrier
 * that gives up sets bit 2 of cabs_diag.status, and every CTA of that kernel
 * leaves it (the sketch's results are then not valid, but the context and
 * the device stay usable). The paper has no counterpart: this is a control
 * for tests of the bounded waits (a limit of 0 makes a wait give up at its
 * first unsuccessful poll). polls >= 0 sets the limit for kernels enqueued
 * from now on by every context of the process (a captured CUDA graph keeps
 * the limit it was captured with); polls < 0 restores the default,
 * CABS_WAIT_LIMIT_DEFAULT (about a second of polling). ctx must be non-NULL. */
#define CABS_WAIT_LIMIT_DEFAULT 16777216
cabs_status cabs_set_wait_limit(cabs_ctx* ctx, int64_t polls);

/* ------------------------------------------------------- whole sketch */

/* Bytes of device workspace cabs_sketch needs for these parameters. */
cabs_status cabs_workspace_size(const cabs_source* src, const cabs_params* p, size_t* bytes);

/* One CABS sketch (Algorithm 2): pilot draw, gather, sketching and embedding,
 * weighted k-means on both embeddings, snap, follow-up gather and sketching;
 * with CABS_FLAG_ERROR also the relative error of the result, enqueued on the
 * same stream and equal bit for bit to what cabs_error returns for the same
 * samples and seed.
 * ws: device workspace of at least cabs_workspace_size() bytes, 256-byte
 * aligned, owned by the caller and not used by anything else until the
 * stream has passed this sketch. Returns CABS_EINVAL for CABS_FLAG_ERROR
 * without out->err, or with err_samples == 0 on an implicit source.
 * The column side of step 3 (k-means and snap of Q) runs on a second,
 * internal stream forked from `stream` and joined back before the follow-up
 * gather; the library creates one such stream and two events per (device,
 * caller stream) it is given and keeps them until the process exits, so a
 * caller should reuse its streams rather than create one per call. */
cabs_status cabs_sketch(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p,
                        void* ws, size_t ws_bytes, cabs_stream stream, const cabs_result* out);

/* `count` independent sketches of different sizes in one call. Member i uses
 * src[i], p[i], out[i] and the workspace slice ws + ws_offsets[i] (host array
 * of byte offsets, each 256-aligned, slices of cabs_workspace_size bytes).
 * Members are scheduled largest-first over `lanes` (1..16; 0 = the lanes
 * cabs_autotune chose for this context, else 8) internal streams
 * forked from and joined back to `stream`; with CUDA graphs enabled
 * (use_graph != 0) the launch sequence of the batch is captured once per
 * distinct batch layout and replayed. Results are bit-identical to running
 * each member alone with cabs_sketch. */
cabs_status cabs_sketch_batched(cabs_ctx* ctx, int32_t count, const cabs_source* src,
                                const cabs_params* p, void* ws, const size_t* ws_offsets,
                                const cabs_result* out, int32_t lanes, int32_t use_graph,
                                cabs_stream stream);

/* ------------------------------------------------------------ launch shapes
 *
 * The paper has no counterpart: these choose how the kernels split their work
 * over the GPU, never what they compute. Every choice gives results bit-
 * identical to the defaults (each output keeps its summation order). A
 * context keeps one cabs_tune per shape bucket -- (prec, ceil(k2 / 32),
 * floor(log2(m + n))) -- which cabs_sketch, cabs_sketch_batched and the
 * serving loop use for every sketch of that bucket; buckets without an entry
 * use the defaults. cabs_autotune fills the table from timed trials. */
typedef struct {
  int32_t extrap_tn;    /* CUDA-core extrapolation GEMMs (C V_w, R^T U_w; FP32 and
                         * FP64 modes, the TF32 / BF16 modes run them on tensor
                         * cores): output columns per thread, 16 extrap_tn per CTA:
                         * 2, 4 or 8 (8 in FP32 only); 0 = default (8 FP32, 4 FP64) */
  int32_t gather_rows;  /* dense column gather: rows of A per warp in flight: 2, 4 or
                         * 8; 0 = default (4) */
  int32_t assign_bn;    /* TF32 / BF16 k-means assignment: centres per tensor-core
                         * column block, 128 or 256 (128 always for TF32 widths above
                         * 128); 0 = default (256) */
  int32_t reserved;     /* 0 */
} cabs_tune;

/* Sets (t != NULL) or removes (t == NULL) the entry of the bucket of (prec, k2,
 * m, n). CABS_EINVAL for a value outside the ranges above. */
cabs_status cabs_tune_set(cabs_ctx* ctx, int32_t prec, int32_t k2, int64_t m, int64_t n, const cabs_tune* t);
/* The entry in force for (prec, k2, m, n): the bucket's, else the defaults
 * (all fields 0). *found (may be NULL) is 1 for a bucket entry. */
cabs_status cabs_tune_get(cabs_ctx* ctx, int32_t prec, int32_t k2, int64_t m, int64_t n, cabs_tune* t,
                          int32_t* found);
/* Writes the table and the tuned lanes to a text file (one line per bucket:
 * "bucket prec kb sb extrap_tn gather_rows assign_bn"; a "lanes L" line), or
 * replaces the context's table with a file's. CABS_EINVAL for an unreadable,
 * unwritable or malformed file (the table is then unchanged). */
cabs_status cabs_tune_save(cabs_ctx* ctx, const char* path);
cabs_status cabs_tune_load(cabs_ctx* ctx, const char* path);
/* Autotuner. For every shape bucket among the `count` members (as for
 * cabs_sketch_batched: their sources, parameters, workspace slices and
 * outputs, which it overwrites), times one representative member's whole
 * sketch on `stream` under each candidate launch shape -- coordinate descent
 * over extrap_tn, gather_rows and assign_bn, the fastest of 5 runs per
 * candidate, a change kept only if it is at least 2 % faster -- and stores
 * the winner in the table. Then it times the whole batch (no graph) at 4, 8,
 * 12 and 16 lanes and keeps the fastest for cabs_sketch_batched with lanes
 * == 0. *lanes_out (may be NULL) receives it. Synchronises `stream`; takes
 * a few seconds for a batch of hundreds of members. */
cabs_status cabs_autotune(cabs_ctx* ctx, int32_t count, const cabs_source* src, const cabs_params* p, void* ws,
                          const size_t* ws_offsets, const cabs_result* out, cabs_stream stream,
                          int32_t* lanes_out);

/* Relative Frobenius error |A - U diag(S) V^T|_F / |A|_F (Section 5).
 * samples == 0: exact, over every entry (dense sources only; FP64 sums of
 * per-tile partial sums). samples > 0: over `samples` entries drawn with
 * replacement by Philox key (seed, 2), counter (t, 0, 0, 0): row = hi64(w0 m),
 * column = hi64(w1 n). U (m x k), S (k), V (n x k) as produced by cabs_sketch.
 * ws: device workspace of cabs_error_workspace_size() bytes.
 * *rel_fro is written on the host, so this call synchronises `stream`. */
cabs_status cabs_error_workspace_size(const cabs_source* src, const cabs_params* p,
                                      int64_t samples, size_t* bytes);
cabs_status cabs_error(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p,
                       const cabs_result* res, int64_t samples, uint64_t seed, void* ws,
                       size_t ws_bytes, cabs_stream stream, double* rel_fro);

/* The error of cabs_error, for callers that cannot allocate device
 * memory when they need it: code running inside another framework's memory
 * pool that forbids cudaMalloc/cudaFree during a step, or programs that
 * reserve all device memory up front and have no workspace to hand out. It
 * takes no workspace and calls no allocating routine. Its products
 * U diag(S) V^T are FP64 in FP64 mode and FP32 CUDA-core products in every
 * other mode: in FP64 and FP32 modes it returns cabs_error's value (to
 * rounding, 1e-9 relative); in TF32 and BF16 modes on a dense FP32 A, where
 * cabs_error forms the products on tensor cores from TF32 / BF16 operands,
 * it returns the FP32-mode value for the same factors, within 1e-3 relative
 * of cabs_error's (the tensor-core residual's bound against the exact error). The paper has no
 * counterpart; this is a service of the library. Its scratch is one fixed
 * file-scope device array (about 256 KiB on every device that loads libcabs,
 * held until the process exits). Limits: the exact error (samples == 0,
 * dense source) takes m <= 1,048,576 rows and returns CABS_EINVAL beyond; the
 * sampled error takes any sample count. The first call on a device looks up
 * the array's address with that device current: make it before any CUDA
 * stream capture starts. Every call shares the array and leaves its contents
 * behind; calls whose kernels overlap on the GPU (other streams or threads)
 * race on it and may return wrong values. Synchronises `stream`. */
cabs_status cabs_error_noalloc(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p,
                               const cabs_result* res, int64_t samples, uint64_t seed, cabs_stream stream,
                               double* rel_fro);

/* ------------------------------------------------ hot-path steps, one by one */

/* Step a1, Algorithm 2 step 1: k distinct uniform indices from [0, N).
 * Partial Fisher-Yates over a virtual identity array; step i swaps positions
 * i and i + hi64(r_i (N - i)), r_i = word 0 of Philox4x64-10 with counter
 * (i, 0, 0, 0) and key (seed, tag). Tags: 0 rows, 1 columns.
 * d_drawn (k, draw order) and d_sorted (k, ascending) are device int32.
 * 0 <= k <= min(N, 4096), N < 2^31. */
cabs_status cabs_draw_indices(cabs_ctx* ctx, uint64_t seed, int32_t tag, int64_t N, int32_t k,
                              int32_t* d_drawn, int32_t* d_sorted, cabs_stream stream);

/* Steps a2 / a7, Algorithm 2 steps 1 and 3: C = A[:, cols] (m x k_c, ld k_c),
 * Rt = A[rows, :]^T (n x k_r, ld k_r), W = A[rows, cols] (k_r x k_c, FP64).
 * C and Rt are elem of `prec`. Any of C, Rt, W may be NULL to skip it (W
 * needs C). Dense entries are copied exactly; RBF entries are generated in
 * elem. W equals C[rows, :] and Rt[cols, :]^T bit for bit. Indices are
 * expected in [0, m) and [0, n); the kernels clamp any that are not, so a bad
 * index never reads outside A, X or Y. */
cabs_status cabs_gather(cabs_ctx* ctx, const cabs_source* src, int64_t m, int64_t n,
                        const int32_t* d_rows, int32_t k_r, const int32_t* d_cols, int32_t k_c,
                        int32_t prec, void* C, void* Rt, double* W, cabs_stream stream);

/* Steps a3 / a4 / a8, Section 4.1 (sketching routine) and Algorithm 2 step 2.
 * SVD W = U_w Sigma_w V_w^T (k x k, k = k_r = k_c) to FP64 accuracy in every
 * mode (an FP32 one-sided Jacobi refined in FP64; an FP64 Jacobi when the
 * refinement does not converge), truncation to
 * sigma_i > max(trunc_rtol, k 2^-52) sigma_1, extrapolation a = C V_w
 * (m x k), b = Rt U_w (n x k) -- FP64 in the FP64 mode, FP32 in the FP32
 * mode, three TF32 tensor-core products with FP32 accumulation in the TF32
 * and BF16 modes -- column norms N_c, N_r, scale S (per cabs_core), then
 *   embed == 0: out1 = U = a N_c^-1, out2 = V = b N_r^-1       (factors)
 *   embed != 0: out1 = P = U S^1/2,  out2 = Q = V S^1/2        (embeddings)
 * out1 (m x k) and out2 (n x k) are elem, ld k; S (k, FP64); columns and S
 * entries beyond the kept rank are zero. d_rank (device int32, may be NULL)
 * receives the kept rank; d_sweeps (may be NULL) the Jacobi sweep count;
 * d_sig / d_Uw / d_Vw (may be NULL) receive Sigma_w (k, descending) and
 * U_w, V_w (k x k, row-major). ws: cabs_sketching_workspace_size() bytes. */
cabs_status cabs_sketching_workspace_size(int64_t m, int64_t n, int32_t k, int32_t prec, size_t* bytes);
cabs_status cabs_sketching(cabs_ctx* ctx, int64_t m, int64_t n, int32_t k, int32_t prec, int32_t core,
                      double trunc_rtol, const void* C, const void* Rt, const double* W,
                      int32_t embed, void* out1, double* S, void* out2, int32_t* d_rank,
                      int32_t* d_sweeps, double* d_sig, double* d_Uw, double* d_Vw, void* ws,
                      size_t ws_bytes, cabs_stream stream);

/* Step a5, Section 3.2 Eq. wkmeans and Algorithm 2 step 3: `iters` Lloyd
 * iterations on the M points X (M x d, elem, ld d) with weights
 * w_l = |X_l|^upsilon_pow (0^0 = 1), from centres X[init_rows[0..k2)].
 * Assign: lowest-index argmin of squared distance; update: weighted mean of
 * the members, an empty cluster keeps its centre.
 * d_labels: iters x M int32 (every iteration's assignment) or NULL;
 * d_centres: k2 x d elem, receives the final centres (after `iters` updates);
 * d_energy: iters doubles (weighted encoding error of each assignment) or NULL;
 * d_T: max cluster size of the last assignment (int32) or NULL.
 * FP64 mode computes distances by direct differences; FP32 by the expansion
 * |z|^2 - 2 x.z on CUDA cores; TF32/BF16 on tensor cores with an FP32
 * re-check of near ties. ws: cabs_kmeans_workspace_size() bytes. */
cabs_status cabs_kmeans_workspace_size(int64_t M, int32_t d, int32_t k2, int32_t iters, int32_t prec,
                                       size_t* bytes);
cabs_status cabs_kmeans(cabs_ctx* ctx, const void* X, int64_t M, int32_t d, const int32_t* d_init_rows,
                        int32_t k2, int32_t iters, int32_t prec, float upsilon_pow, int32_t* d_labels,
                        void* d_centres, double* d_energy, int32_t* d_T, void* ws, size_t ws_bytes,
                        cabs_stream stream);

/* Step a6, Section 3.2 (each centre replaced by its closest in-sample point):
 * centres Z (k2 x d, elem) taken in index order, each picks the nearest row
 * of X (M x d, elem) not yet picked, ties to the lowest row index; distances
 * by direct differences in elem. In the BF16 and TF32 modes (k2 <= 256) the
 * candidates are first ranked by |x|^2 - 2 x.z on tensor cores, and each
 * centre's 32 best are re-ranked by the same direct FP32 distance as in FP32
 * mode before the walk.
 * d_order (k2, pick order) and d_sorted (k2, ascending) are device int32.
 * ws: cabs_snap_workspace_size() bytes. */
cabs_status cabs_snap_workspace_size(int64_t M, int32_t d, int32_t k2, int32_t prec, size_t* bytes);
cabs_status cabs_snap(cabs_ctx* ctx, const void* X, int64_t M, int32_t d, const void* Z, int32_t k2,
                      int32_t prec, int32_t* d_order, int32_t* d_sorted, void* ws, size_t ws_bytes,
                      cabs_stream stream);

/* Section 5, follow-up variant (f): the k2 rows of X (M x d, elem) with the
 * largest squared norm, summed in dimension order with one rounding per
 * multiply and per add (so FP64 keys match a sequential FP64 sum), ties to
 * the lower row index. d_sorted (k2, ascending) is device int32.
 * 1 <= k2 <= M, M < 2^31. ws: cabs_threshold_workspace_size() bytes. */
cabs_status cabs_threshold_workspace_size(int64_t M, size_t* bytes);
cabs_status cabs_threshold(cabs_ctx* ctx, const void* X, int64_t M, int32_t d, int32_t k2, int32_t prec,
                           int32_t* d_sorted, void* ws, size_t ws_bytes, cabs_stream stream);

/* Supplementary Section 3 (orthogonalisation of the sketching output):
 * rewrites U diag(S) V^T as X diag(s) Y^T with orthonormal columns in X and
 * Y, in O((m + n) k^2): U = U_0 Sigma_0 V_0^T (thin SVD, here from the Gram
 * matrix U^T U), then the SVD of Sigma_0 V_0^T diag(S) V^T = U_1 Sigma_1 V_1^T
 * (reduced to k x k through V^T V), X = U_0 U_1, s = diag(Sigma_1), Y = V_1.
 * U (m x k), V (n x k): elem (FP64 for CABS_PREC_FP64, else FP32), ld k,
 * device; S (k, FP64, device). Outputs X (m x k), Y (n x k) elem, ld k, and
 * s (k, FP64, descending) on the device; components with
 * s_i <= max(trunc_rtol, k 2^-52) s_1, and directions in which U or V is
 * numerically singular (a Gram eigenvalue at or below k 2^-52, or 2^-30 for
 * FP32, of the largest), are dropped: zero columns and zero s entries beyond
 * the kept rank, which goes to d_rank (device int32, may be NULL).
 * Orthogonality of X, Y: near 1e-13 (FP64) and 1e-6 (FP32) times
 * cond(U)^2, cond(V)^2. X, Y must not overlap U, V. 1 <= k <= CABS_MAX_K,
 * m, n >= 1. ws: cabs_orthogonalize_workspace_size() bytes (256-aligned). */
cabs_status cabs_orthogonalize_workspace_size(int64_t m, int64_t n, int32_t k, int32_t prec, size_t* bytes);
cabs_status cabs_orthogonalize(cabs_ctx* ctx, int64_t m, int64_t n, int32_t k, int32_t prec, double trunc_rtol,
                               const void* U, const double* S, const void* V, void* X, double* s, void* Y,
                               int32_t* d_rank, void* ws, size_t ws_bytes, cabs_stream stream);

/* Section 2.2, Algorithm 1 (Bilateral Resampling CUR) as Sketch-CUR:
 * independent uniform base samplings I^b_r, I^b_c (kb each; the pilot draw,
 * Philox tags 0 and 1) and target samplings I^t_r, I^t_c (kt each, tags 4 and
 * 5; Section 5 compares at kt = 3 kb). C = A[:, I^b_c], R = A[I^b_r, :],
 * C_bar = A[I^t_r, I^b_c], R_bar = A[I^b_r, I^t_c], M = A[I^t_r, I^t_c],
 * U* = C_bar^+ M R_bar^+ (FP64; pseudo-inverses truncated at
 * sigma_i <= max(trunc_rtol, K 2^-52) sigma_1, K = max(kb, kt)).
 * A ~ C U* R = U diag(S) V^T with U = C U*, S = 1, V = R^T. */
typedef struct {
  int64_t m, n;       /* A is m x n */
  int32_t kb, kt;     /* base and target samples per side, 1..min(m, n, CABS_MAX_K) */
  uint64_t seed;      /* Philox key word 0 of all four draws */
  int32_t prec;       /* cabs_prec: elem type of U, V (FP64, else FP32) */
  double trunc_rtol;
} cabs_cur_params;

typedef struct {
  void* U;            /* elem, m x kb (ld kb): C U* */
  double* S;          /* kb: ones */
  void* V;            /* elem, n x kb (ld kb): R^T */
  double* Ustar;      /* kb x kb FP64 row-major, or NULL */
  int32_t *rows_b, *cols_b;   /* kb each, ascending */
  int32_t *rows_t, *cols_t;   /* kt each, ascending */
  int32_t* ranks;     /* 8 (or NULL): kept ranks of C_bar^+ and R_bar^+; the FP32
                         Jacobi sweeps and the FP64 refinement iterations (-1:
                         FP64 Jacobi fallback) of their SVDs; the SVD status
                         bits (as cabs_diag.status); one reserved */
} cabs_cur_result;

cabs_status cabs_sketch_cur_workspace_size(const cabs_source* src, const cabs_cur_params* p, size_t* bytes);
cabs_status cabs_sketch_cur(cabs_ctx* ctx, const cabs_source* src, const cabs_cur_params* p, void* ws,
                            size_t ws_bytes, cabs_stream stream, const cabs_cur_result* out);

/* ----------------------------------------------------------- profiling */

/* Per-kernel device timing: while enabled, CUDA events are recorded on the
 * launching stream around every kernel launch that libcabs issues in this
 * process (not inside a CUDA graph capture). Off by default; process-wide. */
cabs_status cabs_profile_enable(cabs_ctx* ctx, int32_t on);
/* Waits for the timed launches, then writes up to `max` rows, one per kernel
 * name: names (max rows of name_len chars, NUL-terminated), launch counts and
 * summed device milliseconds. Returns the number of rows written; reset != 0
 * clears the accumulated totals. */
int32_t cabs_profile_read(cabs_ctx* ctx, char* names, int32_t name_len, int64_t* launches, double* total_ms,
                          int32_t max, int32_t reset);
/* Number of kernel launches libcabs has issued in this process; each replay
 * of a captured batch graph counts the kernels the graph holds. Launches made
 * while a graph is being captured are not counted until it is replayed.
 * Profiling (cabs_profile_enable) skips captured launches. */
int64_t cabs_launch_count(void);

/* ------------------------------------------------------------- serving */

/* Continuous-batching request loop on one device. The caller hands over an
 * HBM arena (device memory, `arena_bytes`, owned by the caller and not
 * touched by it until cabs_serve_stop returns); each request's workspace and
 * its resident results are carved from the arena. A request is admitted when
 * a slot is free and its footprint fits in the unused arena; requests on the
 * device run concurrently on up to `max_slots` streams. */
cabs_status cabs_serve_start(cabs_ctx* ctx, void* arena, size_t arena_bytes, int32_t max_slots);
/* Queues one request (copies *src and *p). The request's result buffers are
 * resident in the arena until cabs_serve_release. Thread-safe. */
cabs_status cabs_serve_submit(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p,
                              uint64_t* ticket);
/* Waits up to timeout_ms (0 = poll) for a request. On CABS_OK, *res points
 * into the arena (device pointers valid until release) and *latency_ms holds
 * submit-to-completion time. CABS_EBUSY: not finished yet. */
cabs_status cabs_serve_poll(cabs_ctx* ctx, uint64_t ticket, cabs_result* res, double* latency_ms,
                            int32_t timeout_ms);
/* Device-side interval of a finished request: *start_ms and *end_ms are the
 * times (ms since cabs_serve_start) at which its slot stream reached the
 * request's first and passed its last kernel, from CUDA events on that
 * stream. Two requests whose intervals intersect had work on the GPU at the
 * same time. CABS_EBUSY while the request is queued or running,
 * CABS_ENOTFOUND after cabs_serve_release. The paper has no counterpart. */
cabs_status cabs_serve_times(cabs_ctx* ctx, uint64_t ticket, double* start_ms, double* end_ms);

/* Frees a finished request's resident results. */
cabs_status cabs_serve_release(cabs_ctx* ctx, uint64_t ticket);
/* Stops admitting, waits for requests on the device, joins the loop. */
cabs_status cabs_serve_stop(cabs_ctx* ctx);

#if defined(__GNUC__)
#pragma GCC visibility pop
#endif

#ifdef __cplusplus
}
#endif
#endif /* CABS_H */
