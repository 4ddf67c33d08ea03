// Orthogonalisation of a sketch (supplementary Section 3): U diag(S) V^T,
// with U (m x k) and V (n x k) not orthonormal, rewritten as
// X diag(s) Y^T with orthonormal X, Y in O((m + n) k^2).
//
// The supplementary text takes the thin SVD U = U_0 Sigma_0 V_0^T and then
// the SVD of the k x n matrix B = Sigma_0 V_0^T diag(S) V^T = U_1 Sigma_1 V_1^T,
// giving X = U_0 U_1, s = Sigma_1, Y = V_1. Here both tall factors reach
// the k x k level through their Gram matrices, the only steps that read them:
//
//  1. gram_kernel / gram_reduce_kernel: G_u = U^T U and G_v = V^T V. A CTA
//     owns one tile of the upper triangle and a chunk of a few hundred rows;
//     its threads accumulate an 8 x 8 (FP32) or 4 x 4 (FP64) register tile
//     over the chunk, and the chunk partials are summed in FP64 in chunk
//     order (deterministic). Short FP32 chains keep the error of G near
//     2^-24 (chunk / sqrt(m)) relative.
//  2. G_u = E_u Lambda_u E_u^T (the k x k SVD of a symmetric PSD matrix), so
//     U = (U E_u Lambda_u^-1/2) (Lambda_u^1/2 E_u^T): U_0 = U E_u Lambda_u^-1/2,
//     Sigma_0 = Lambda_u^1/2, V_0 = E_u. Likewise V = Q_v R_v with
//     Q_v = V E_v Lambda_v^-1/2, R_v = Lambda_v^1/2 E_v^T. Eigenvalues at or
//     below the Gram's resolution (Lambda_i <= tol Lambda_1) are dropped.
//  3. B = M Q_v^T with the k x k matrix M = Sigma_0 V_0^T diag(S) R_v^T, so
//     the SVD of B is that of M: M = U_1 Sigma_1 Z^T and V_1 = Q_v Z.
//  4. X = U (E_u Lambda_u^-1/2 U_1), Y = V (E_v Lambda_v^-1/2 Z): one k x k
//     FP64 product each, then one tall product each on CUDA cores.
// The k x k SVDs are the FP64-accurate SVD of the sketching routine.
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"
#include "svd.cuh"

namespace cabs {
namespace {

constexpr int kGK = 16;         // rows staged per step
constexpr int kGramCtas = 608;  // 4 x 152: target CTAs of one Gram launch

template <typename T>
struct GramTile {
  static constexpr int TT = sizeof(T) == 4 ? 8 : 4;  // register tile per thread
  static constexpr int BT = 16 * TT;                 // output tile per CTA
};

__host__ __device__ inline int gram_tiles(int K, int BT) {
  const int nt = (K + BT - 1) / BT;
  return nt * (nt + 1) / 2;
}

template <typename T>
void gram_split(int64_t M, int K, int& chunks, int64_t& rows) {
  const int tri = gram_tiles(K, GramTile<T>::BT);
  const int64_t max_chunks = (M + kGK - 1) / kGK;
  const int64_t want = std::max<int64_t>(1, std::min<int64_t>(max_chunks, (kGramCtas + tri - 1) / tri));
  rows = ((M + want - 1) / want + kGK - 1) / kGK * kGK;
  chunks = (int)((M + rows - 1) / rows);
}

template <typename T>
size_t gram_part_elems(int64_t M, int K) {
  int chunks;
  int64_t rows;
  gram_split<T>(M, K, chunks, rows);
  const size_t bt = GramTile<T>::BT;
  return (size_t)chunks * gram_tiles(K, GramTile<T>::BT) * bt * bt;
}

// Tile t of the upper triangle (row-major over tile rows) -> (bi, bj), bi <= bj.
__device__ __forceinline__ void tri_tile(int t, int nt, int& bi, int& bj) {
  bi = 0;
  while (t >= nt - bi) {
    t -= nt - bi;
    ++bi;
  }
  bj = bi + t;
}

template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const T* __restrict__ X, long long M, int K, long long rows,
                                                  T* __restrict__ part) {
  constexpr int TT = GramTile<T>::TT, BT = GramTile<T>::BT;
  constexpr int L = BT * kGK / 256;  // elements each thread stages per operand and step
  __shared__ __align__(16) T As[2][kGK][BT + 4];
  __shared__ __align__(16) T Bs[2][kGK][BT + 4];
  const int nt = (K + BT - 1) / BT;
  int bi, bj;
  tri_tile(blockIdx.x, nt, bi, bj);
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const long long r_begin = (long long)blockIdx.y * rows;
  const long long r_end = min(M, r_begin + rows);
  T acc[TT][TT];
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) acc[i][j] = T(0);
  T ra[L], rb[L];
  auto load = [&](long long r0) {
#pragma unroll
    for (int e = 0; e < L; ++e) {
      const int idx = tid + 256 * e;
      const int r = idx / BT, c = idx - r * BT;
      const long long gr = r0 + r;
      const int ca = bi * BT + c, cb = bj * BT + c;
      const bool in = gr < r_end;
      ra[e] = (in && ca < K) ? X[gr * K + ca] : T(0);
      rb[e] = (in && cb < K) ? X[gr * K + cb] : T(0);
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < L; ++e) {
      const int idx = tid + 256 * e;
      const int r = idx / BT, c = idx - r * BT;
      As[buf][r][c] = ra[e];
      Bs[buf][r][c] = rb[e];
    }
  };
  load(r_begin);
  store(0);
  __syncthreads();
  int buf = 0;
  for (long long r0 = r_begin; r0 < r_end; r0 += kGK) {
    const bool more = r0 + kGK < r_end;
    if (more) load(r0 + kGK);
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      T a[TT], b[TT];
#pragma unroll
      for (int i = 0; i < TT; ++i) a[i] = As[buf][kk][ty * TT + i];
#pragma unroll
      for (int j = 0; j < TT; ++j) b[j] = Bs[buf][kk][tx * TT + j];
#pragma unroll
      for (int i = 0; i < TT; ++i)
#pragma unroll
        for (int j = 0; j < TT; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  T* out = part + ((size_t)blockIdx.y * gridDim.x + blockIdx.x) * BT * BT;
#pragma unroll
  for (int i = 0; i < TT; ++i)
#pragma unroll
    for (int j = 0; j < TT; ++j) out[(size_t)(ty * TT + i) * BT + tx * TT + j] = acc[i][j];
}

// G[i][j] = G[j][i] = sum over chunks, in chunk order, of the partials.
template <typename T>
__global__ void gram_reduce_kernel(const T* __restrict__ part, int chunks, int K, double* __restrict__ G) {
  constexpr int BT = GramTile<T>::BT;
  const int nt = (K + BT - 1) / BT, tri = nt * (nt + 1) / 2;
  const long long total = (long long)tri * BT * BT;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int t = (int)(e / (BT * BT));
    const int w = (int)(e - (long long)t * BT * BT);
    const int a = w / BT, b = w - a * BT;
    int bi, bj;
    tri_tile(t, nt, bi, bj);
    const int i = bi * BT + a, j = bj * BT + b;
    if (i >= K || j >= K || (bi == bj && a > b)) continue;
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)part[((size_t)c * tri + t) * BT * BT + w];
    G[(size_t)i * K + j] = s;
    G[(size_t)j * K + i] = s;
  }
}

// From the eigenvalues (descending) and kept ranks of G_u and G_v:
// su = Lambda_u^1/2, isu = Lambda_u^-1/2 (zero beyond the rank), same for v.
__global__ void orth_scales_kernel(int k, const double* __restrict__ lu, const int* __restrict__ ru,
                                   const double* __restrict__ lv, const int* __restrict__ rv, double* __restrict__ su,
                                   double* __restrict__ isu, double* __restrict__ sv, double* __restrict__ isv) {
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    const bool ku = i < *ru && lu[i] > 0.0, kv = i < *rv && lv[i] > 0.0;
    su[i] = ku ? sqrt(lu[i]) : 0.0;
    isu[i] = ku ? 1.0 / sqrt(lu[i]) : 0.0;
    sv[i] = kv ? sqrt(lv[i]) : 0.0;
    isv[i] = kv ? 1.0 / sqrt(lv[i]) : 0.0;
  }
}

// k x k FP64: C[i][j] = a_i b_j sum_l op(A)[i][l] d_l op(B)[l][j], op(X) = X
// or X^T; a, b, d may be NULL (ones). Row-major operands. 16 x 16 outputs per
// CTA, one per thread, l in ascending order.
__global__ void __launch_bounds__(256) kk_gemm_kernel(int k, const double* __restrict__ A, int transA,
                                                      const double* __restrict__ d, const double* __restrict__ B,
                                                      int transB, const double* __restrict__ a,
                                                      const double* __restrict__ b, double* __restrict__ C) {
  __shared__ double As[16][17], Bs[16][17];
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int l0 = 0; l0 < k; l0 += 16) {
    // As[ty][tx] = op(A)[blockIdx.y*16 + ty][l0 + tx] * d[l0 + tx]
    const int ai = blockIdx.y * 16 + ty, al = l0 + tx;
    double av = 0.0;
    if (ai < k && al < k) av = transA ? A[(size_t)al * k + ai] : A[(size_t)ai * k + al];
    if (d && al < k) av *= d[al];
    As[ty][tx] = av;
    const int bl = l0 + ty, bj = blockIdx.x * 16 + tx;
    double bv = 0.0;
    if (bl < k && bj < k) bv = transB ? B[(size_t)bj * k + bl] : B[(size_t)bl * k + bj];
    Bs[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) acc = fma(As[ty][l], Bs[l][tx], acc);
    __syncthreads();
  }
  if (i < k && j < k) {
    double v = acc;
    if (a) v *= a[i];
    if (b) v *= b[j];
    C[(size_t)i * k + j] = v;
  }
}

// Small FP64 product C (M x N, ld ldc) = op(A) diag(d) op(B), op(A) M x K and
// op(B) K x N; op(X) = X or X^T of a row-major X with leading dimension ld;
// d may be NULL. 16 x 16 outputs per CTA, l in ascending order.
__global__ void __launch_bounds__(256) small_gemm_kernel(int M, int N, int K, const double* __restrict__ A, int lda,
                                                         int transA, const double* __restrict__ d,
                                                         const double* __restrict__ B, int ldb, int transB,
                                                         double* __restrict__ C, int ldc) {
  __shared__ double As[16][17], Bs[16][17];
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  const int i = blockIdx.y * 16 + ty, j = blockIdx.x * 16 + tx;
  double acc = 0.0;
  for (int l0 = 0; l0 < K; l0 += 16) {
    const int al = l0 + tx;
    double av = 0.0;
    if (i < M && al < K) av = transA ? A[(size_t)al * lda + i] : A[(size_t)i * lda + al];
    if (d && al < K) av *= d[al];
    As[ty][tx] = av;
    const int bl = l0 + ty;
    double bv = 0.0;
    if (bl < K && j < N) bv = transB ? B[(size_t)j * ldb + bl] : B[(size_t)bl * ldb + j];
    Bs[ty][tx] = bv;
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) acc = fma(As[ty][l], Bs[l][tx], acc);
    __syncthreads();
  }
  if (i < M && j < N) C[(size_t)i * ldc + j] = acc;
}

// Zero s beyond the kept rank; column masks for the tail products.
__global__ void orth_final_kernel(int k, const int* __restrict__ rank, double* __restrict__ s,
                                  double* __restrict__ mask, int* __restrict__ rank_out) {
  const int r = *rank;
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    if (i >= r) s[i] = 0.0;
    mask[i] = i < r ? 1.0 : 0.0;
  }
  if (threadIdx.x == 0 && rank_out) *rank_out = r;
}

struct OrthWs {
  SvdWs svd;
  double *Gu, *Gv, *lu, *lv, *Eu, *Ev, *Fu, *Fv, *Mk, *P, *Z, *Tu, *Tv;
  double *su, *isu, *sv, *isv, *mask, *part_x;
  void* gpart;
  int *ru, *rv, *rk, *sweeps, *refine, *status;
};

OrthWs carve_orth(Carve& cv, int64_t m, int64_t n, int k, bool f64) {
  OrthWs w;
  w.svd = carve_svd(cv, k);
  const size_t kk = (size_t)k * k;
  w.Gu = cv.take<double>(kk);
  w.Gv = cv.take<double>(kk);
  w.Eu = cv.take<double>(kk);
  w.Ev = cv.take<double>(kk);
  w.Fu = cv.take<double>(kk);
  w.Fv = cv.take<double>(kk);
  w.Mk = cv.take<double>(kk);
  w.P = cv.take<double>(kk);
  w.Z = cv.take<double>(kk);
  w.Tu = cv.take<double>(kk);
  w.Tv = cv.take<double>(kk);
  w.lu = cv.take<double>(k);
  w.lv = cv.take<double>(k);
  w.su = cv.take<double>(k);
  w.isu = cv.take<double>(k);
  w.sv = cv.take<double>(k);
  w.isv = cv.take<double>(k);
  w.mask = cv.take<double>(k);
  w.part_x = cv.take<double>((size_t)extrap_row_blocks(std::max(m, n), f64) * k);
  const size_t ge = f64 ? std::max(gram_part_elems<double>(m, k), gram_part_elems<double>(n, k))
                        : std::max(gram_part_elems<float>(m, k), gram_part_elems<float>(n, k));
  w.gpart = f64 ? (void*)cv.take<double>(ge) : (void*)cv.take<float>(ge);
  w.ru = cv.take<int>(1);
  w.rv = cv.take<int>(1);
  w.rk = cv.take<int>(1);
  w.sweeps = cv.take<int>(1);
  w.refine = cv.take<int>(1);
  w.status = cv.take<int>(1);
  return w;
}

template <typename T>
cabs_status gram(const T* X, int64_t M, int K, T* part, double* G, cudaStream_t stream) {
  int chunks;
  int64_t rows;
  gram_split<T>(M, K, chunks, rows);
  const int tri = gram_tiles(K, GramTile<T>::BT);
  CABS_LAUNCH(stream, "gram_kernel", gram_kernel<T><<<dim3(tri, chunks), 256, 0, stream>>>(X, M, K, rows, part));
  const long long total = (long long)tri * GramTile<T>::BT * GramTile<T>::BT;
  const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)sm_count() * 4);
  CABS_LAUNCH(stream, "gram_reduce_kernel", gram_reduce_kernel<T><<<blocks, 256, 0, stream>>>(part, chunks, K, G));
  return CABS_OK;
}

template <typename T>
cabs_status orth_typed(int64_t m, int64_t n, int k, double trunc_rtol, const T* U, const double* S, const T* V, T* X,
                       double* s, T* Y, int* d_rank, int* d_status, void* ws, size_t ws_bytes, cudaStream_t stream) {
  Carve cv(ws, ws_bytes);
  OrthWs w = carve_orth(cv, m, n, k, sizeof(T) == 8);
  if (!cv.fits()) {
    set_error("orthogonalisation workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  if (!d_status) {
    d_status = w.status;
    if (cudaMemsetAsync(d_status, 0, sizeof(int), stream) != cudaSuccess) return check_cuda("orth status clear");
  }
  // Gram eigenvalues below the resolution of G (relative to Lambda_1) are
  // dropped: k 2^-52 in FP64, 2^-30 for FP32 factors (directions of U or V
  // below 2^-15 of their largest singular value).
  const double tol_g = sizeof(T) == 8 ? 0.0 : 9.313225746154785e-10;
  CABS_TRY(gram<T>(U, m, k, (T*)w.gpart, w.Gu, stream));
  CABS_TRY(gram<T>(V, n, k, (T*)w.gpart, w.Gv, stream));
  const double res = sizeof(T) == 8 ? 0.0 : kResolveReduced;
  CABS_TRY(launch_svd(w.Gu, k, tol_g, res, w.lu, w.Fu, w.Eu, w.ru, w.sweeps, w.refine, d_status, w.svd, stream));
  CABS_TRY(launch_svd(w.Gv, k, tol_g, res, w.lv, w.Fv, w.Ev, w.rv, w.sweeps, w.refine, d_status, w.svd, stream));
  CABS_LAUNCH(stream, "orth_scales_kernel",
              orth_scales_kernel<<<1, 256, 0, stream>>>(k, w.lu, w.ru, w.lv, w.rv, w.su, w.isu, w.sv, w.isv));
  // M = Lambda_u^1/2 E_u^T diag(S) E_v Lambda_v^1/2
  CABS_TRY(launch_kk_gemm(k, w.Eu, true, S, w.Ev, false, w.su, w.sv, w.Mk, stream));
  CABS_TRY(launch_svd(w.Mk, k, trunc_rtol, res, s, w.P, w.Z, w.rk, w.sweeps, w.refine, d_status, w.svd, stream));
  CABS_LAUNCH(stream, "orth_final_kernel", orth_final_kernel<<<1, 256, 0, stream>>>(k, w.rk, s, w.mask, d_rank));
  // T_u = E_u Lambda_u^-1/2 U_1, T_v = E_v Lambda_v^-1/2 Z (columns beyond the rank zero)
  CABS_TRY(launch_kk_gemm(k, w.Eu, false, w.isu, w.P, false, nullptr, w.mask, w.Tu, stream));
  CABS_TRY(launch_kk_gemm(k, w.Ev, false, w.isv, w.Z, false, nullptr, w.mask, w.Tv, stream));
  CABS_TRY(launch_extrap_gemm(U, m, k, w.Tu, k, sizeof(T) == 8, X, w.part_x, "extrap_gemm_kernel(X = U T_u)", stream));
  CABS_TRY(launch_extrap_gemm(V, n, k, w.Tv, k, sizeof(T) == 8, Y, w.part_x, "extrap_gemm_kernel(Y = V T_v)", stream));
  return CABS_OK;
}

}  // namespace

size_t gram_ws_bytes(int64_t M, int K, bool elem_f64) {
  const size_t e = elem_f64 ? gram_part_elems<double>(M, K) * sizeof(double) : gram_part_elems<float>(M, K) * sizeof(float);
  return align256(e);
}

cabs_status launch_gram(const void* X, int64_t M, int K, bool elem_f64, void* part, double* G, cudaStream_t stream) {
  if (elem_f64) return gram<double>((const double*)X, M, K, (double*)part, G, stream);
  return gram<float>((const float*)X, M, K, (float*)part, G, stream);
}

cabs_status launch_kk_gemm(int k, const double* A, bool transA, const double* d, const double* B, bool transB,
                           const double* a, const double* b, double* C, cudaStream_t stream) {
  const dim3 g(ceil_div(k, 16), ceil_div(k, 16));
  CABS_LAUNCH(stream, "kk_gemm_kernel",
              kk_gemm_kernel<<<g, 256, 0, stream>>>(k, A, transA ? 1 : 0, d, B, transB ? 1 : 0, a, b, C));
  return CABS_OK;
}

cabs_status launch_small_gemm(int M, int N, int K, const double* A, int lda, bool transA, const double* d,
                              const double* B, int ldb, bool transB, double* C, int ldc, cudaStream_t stream) {
  const dim3 g(ceil_div(N, 16), ceil_div(M, 16));
  CABS_LAUNCH(stream, "small_gemm_kernel",
              small_gemm_kernel<<<g, 256, 0, stream>>>(M, N, K, A, lda, transA ? 1 : 0, d, B, ldb, transB ? 1 : 0, C,
                                                       ldc));
  return CABS_OK;
}

size_t orth_ws_bytes(int64_t m, int64_t n, int k, bool elem_f64) {
  Carve cv;
  carve_orth(cv, m, n, k, elem_f64);
  return cv.used;
}

cabs_status launch_orthogonalize(int64_t m, int64_t n, int k, bool elem_f64, double trunc_rtol, const void* U,
                                 const double* S, const void* V, void* X, double* s, void* Y, int* d_rank,
                                 int* d_status, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (elem_f64)
    return orth_typed<double>(m, n, k, trunc_rtol, (const double*)U, S, (const double*)V, (double*)X, s, (double*)Y,
                              d_rank, d_status, ws, ws_bytes, stream);
  return orth_typed<float>(m, n, k, trunc_rtol, (const float*)U, S, (const float*)V, (float*)X, s, (float*)Y, d_rank,
                           d_status, ws, ws_bytes, stream);
}

}  // namespace cabs
