// The C ABI of libcabs (declared in include/cabs.h): argument checks,
// workspace layout, and the order in which one sketch (Algorithm 2) launches
// the step kernels. No step runs on the host.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "api_internal.cuh"
#include "common.cuh"
#include "kernels.cuh"
#include "profile.cuh"

namespace cabs {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }
const char* last_error() { return g_err.c_str(); }

cabs_status check_cuda(const char* what) {
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    return CABS_ECUDA;
  }
  return CABS_OK;
}

int sm_count() {
  static int cache[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (cache[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

static thread_local int t_sharers = 1;

SharersScope::SharersScope(int sharers) : prev(t_sharers) { t_sharers = sharers < 1 ? 1 : sharers; }
SharersScope::~SharersScope() { t_sharers = prev; }

int coop_grid_cap(int full) { return std::max(16, full / t_sharers); }

static std::atomic<long long> g_wait_limit{CABS_WAIT_LIMIT_DEFAULT};
long long wait_limit() { return g_wait_limit.load(std::memory_order_relaxed); }

DeviceGuard::DeviceGuard(int dev) {
  ok = cudaGetDevice(&prev) == cudaSuccess;
  if (ok && prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
  target = dev;
}
DeviceGuard::~DeviceGuard() {
  if (ok && prev != target) cudaSetDevice(prev);
}

// The BF16 and TF32 modes take the extrapolation products on the tensor
// cores (3 x TF32, FP32-level); FP32 and FP64 keep CUDA-core arithmetic.
static bool tc_extrap_ok(int prec) { return prec == CABS_PREC_BF16 || prec == CABS_PREC_TF32; }

// ------------------------------------------------------------- validation

static bool finite(double x) { return std::isfinite(x); }

cabs_status validate_source(const cabs_source* src, int64_t m, int64_t n) {
  CABS_REQUIRE(src != nullptr, "source is NULL");
  if (src->kind == CABS_SRC_DENSE) {
    CABS_REQUIRE(src->A != nullptr, "dense source: A is NULL");
    CABS_REQUIRE(src->lda >= n, "dense source: lda (%lld) < n (%lld)", (long long)src->lda, (long long)n);
  } else if (src->kind == CABS_SRC_RBF) {
    CABS_REQUIRE(src->X != nullptr && src->Y != nullptr, "rbf source: X or Y is NULL");
    CABS_REQUIRE(src->d >= 1 && src->d <= CABS_MAX_D, "rbf source: d = %d outside [1, %d]", src->d, CABS_MAX_D);
    CABS_REQUIRE(src->sigma > 0.0f && finite(src->sigma), "rbf source: sigma must be positive and finite");
  } else if (src->kind == CABS_SRC_CSR) {
    CABS_REQUIRE(src->row_ptr != nullptr, "csr source: row_ptr is NULL");
    CABS_REQUIRE(src->nnz >= 0, "csr source: nnz < 0");
    CABS_REQUIRE(src->nnz == 0 || (src->col_idx != nullptr && src->A != nullptr),
                 "csr source: col_idx or values are NULL");
  } else {
    CABS_REQUIRE(false, "unknown source kind %d", src->kind);
  }
  (void)m;
  return CABS_OK;
}

cabs_status validate_params(const cabs_params* p) {
  CABS_REQUIRE(p != nullptr, "params is NULL");
  CABS_REQUIRE(p->m >= 1 && p->n >= 1, "m and n must be >= 1");
  CABS_REQUIRE(p->m < (int64_t)INT32_MAX && p->n < (int64_t)INT32_MAX, "m and n must be < 2^31");
  const int64_t mn = std::min(p->m, p->n);
  CABS_REQUIRE(p->k1 >= 1 && p->k1 <= CABS_MAX_K && p->k1 <= mn, "k1 = %d outside [1, min(m, n, %d)]", p->k1,
               CABS_MAX_K);
  CABS_REQUIRE(p->k2 >= 1 && p->k2 <= p->k1, "k2 = %d outside [1, k1]", p->k2);
  CABS_REQUIRE(p->iters >= 0 && p->iters <= CABS_MAX_ITERS, "iters = %d outside [0, %d]", p->iters, CABS_MAX_ITERS);
  CABS_REQUIRE(p->prec >= CABS_PREC_FP64 && p->prec <= CABS_PREC_BF16, "unknown precision %d", p->prec);
  CABS_REQUIRE(p->core == CABS_CORE_PINV || p->core == CABS_CORE_STABILIZED, "unknown core %d", p->core);
  CABS_REQUIRE(finite(p->upsilon_pow), "upsilon_pow must be finite");
  CABS_REQUIRE(finite(p->trunc_rtol) && p->trunc_rtol >= 0.0, "trunc_rtol must be finite and >= 0");
  CABS_REQUIRE((p->flags & ~(CABS_FLAG_FOLLOW_ERR | CABS_FLAG_ERROR | CABS_FLAG_HARD_THRESHOLD | CABS_FLAG_SVD_FORM |
                             CABS_FLAG_LEVERAGE)) == 0,
               "unknown flags 0x%x", p->flags);
  CABS_REQUIRE(!((p->flags & CABS_FLAG_HARD_THRESHOLD) && (p->flags & CABS_FLAG_LEVERAGE)),
               "CABS_FLAG_HARD_THRESHOLD and CABS_FLAG_LEVERAGE exclude each other");
  if (p->flags & CABS_FLAG_ERROR) CABS_REQUIRE(p->err_samples >= 0, "err_samples must be >= 0");
  return CABS_OK;
}

// A sketch that also computes its error needs somewhere to put it, and the
// exact error needs stored entries.
cabs_status validate_error_request(const cabs_source* src, const cabs_params* p, const cabs_result* out) {
  if (!(p->flags & CABS_FLAG_ERROR)) return CABS_OK;
  CABS_REQUIRE(out->err != nullptr, "CABS_FLAG_ERROR needs result.err");
  CABS_REQUIRE(p->err_samples > 0 || src->kind != CABS_SRC_RBF, "the exact error needs stored entries (dense or CSR)");
  return CABS_OK;
}

// -------------------------------------------------------------- workspace

SketchWs carve_sketch(Carve& cv, const cabs_source& src, const cabs_params& p) {
  const size_t eb = elem_bytes(p.prec);
  const int64_t m = p.m, n = p.n;
  const int k1 = p.k1, k2 = p.k2;
  SketchWs w;
  w.pr_drawn = cv.take<int>(k1);
  w.pc_drawn = cv.take<int>(k1);
  w.fr_order = cv.take<int>(k2);
  w.fc_order = cv.take<int>(k2);
  w.C = cv.take<char>((size_t)m * k1 * eb);
  w.Rt = cv.take<char>((size_t)n * k1 * eb);
  w.W = cv.take<double>((size_t)k1 * k1);
  w.P = cv.take<char>((size_t)m * k1 * eb);
  w.Q = cv.take<char>((size_t)n * k1 * eb);
  w.S_pilot = cv.take<double>(k1);
  w.Zr = cv.take<char>((size_t)k2 * k1 * eb);
  w.Zc = cv.take<char>((size_t)k2 * k1 * eb);
  w.diag = cv.take<cabs_diag>(1);
  size_t core_b = std::max(core_ws_bytes(m, n, k1, eb == 8), core_ws_bytes(m, n, k2, eb == 8));
  if (p.flags & CABS_FLAG_SVD_FORM) core_b = std::max(core_b, orth_ws_bytes(m, n, k2, eb == 8));
  if (p.flags & CABS_FLAG_LEVERAGE) core_b = std::max(core_b, orth_ws_bytes(m, n, k1, eb == 8));
  size_t side_r = std::max(kmeans_ws_bytes(m, k1, k2, p.iters, p.prec), snap_ws_bytes(m, k1, k2, p.prec));
  size_t side_c = std::max(kmeans_ws_bytes(n, k1, k2, p.iters, p.prec), snap_ws_bytes(n, k1, k2, p.prec));
  side_r = std::max({side_r, kmeans_ws_bytes(m, k1, k2, 1, p.prec), threshold_ws_bytes(m)});
  side_c = std::max({side_c, kmeans_ws_bytes(n, k1, k2, 1, p.prec), threshold_ws_bytes(n)});
  w.core_bytes = align256(core_b);
  w.side_r_bytes = align256(side_r);
  w.side_c_bytes = align256(side_c);
  w.core = cv.take<char>(w.core_bytes);
  w.side_r = cv.take<char>(w.side_r_bytes);
  w.side_c = cv.take<char>(w.side_c_bytes);
  w.lev_X = w.lev_Y = nullptr;
  w.lev_one = w.lev_s = nullptr;
  if (p.flags & CABS_FLAG_LEVERAGE) {
    w.lev_X = cv.take<char>((size_t)m * k1 * eb);
    w.lev_Y = cv.take<char>((size_t)n * k1 * eb);
    w.lev_one = cv.take<double>(k1);
    w.lev_s = cv.take<double>(k1);
  }
  w.err_out2 = nullptr;
  w.err_ws = nullptr;
  w.err_bytes = 0;
  if (p.flags & CABS_FLAG_ERROR) {
    w.err_out2 = cv.take<double>(2);
    w.err_bytes = align256(error_ws_bytes(src, m, n, k2, p.err_samples, p.prec));
    w.err_ws = cv.take<char>(w.err_bytes);
  }
  return w;
}

size_t sketch_ws_bytes(const cabs_source& src, const cabs_params& p) {
  Carve cv;
  carve_sketch(cv, src, p);
  return cv.used;
}

// err = sqrt(num / den), the same correctly rounded operations as the host
// side of cabs_error.
__global__ void err_finalize_kernel(const double* out2, double* err) {
  if (threadIdx.x == 0) err[0] = out2[1] > 0.0 ? sqrt(out2[0] / out2[1]) : 0.0;
}

__global__ void fill_kernel(double* x, int n, double v) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) x[i] = v;
}

__global__ void diag_clear_kernel(cabs_diag* d) {
  int* p = (int*)d;
  for (size_t i = threadIdx.x; i < sizeof(cabs_diag) / sizeof(int); i += blockDim.x) p[i] = 0;
}

// A second stream per (device, stream) on which a sketch runs its column
// side of step 3 (k-means and snap of Q) while the row side runs on its own
// stream; created on first use, kept until exit. Work issued on one stream is
// serialised, so its side stream serves one sketch at a time; the fork and
// join are event waits, which stream capture turns into graph edges.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

static cabs_status side_stream_of(cudaStream_t main, SideStream& out) {
  static std::mutex mu;
  static std::map<std::pair<int, cudaStream_t>, SideStream> sides;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return check_cuda("cudaGetDevice");
  std::lock_guard<std::mutex> lk(mu);
  SideStream& e = sides[{dev, main}];
  if (!e.s) {
    if (cudaStreamCreateWithFlags(&e.s, cudaStreamNonBlocking) != cudaSuccess) return check_cuda("side stream");
    if (cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&e.join, cudaEventDisableTiming) != cudaSuccess)
      return check_cuda("side stream events");
  }
  out = e;
  return CABS_OK;
}

constexpr int kTagLevRows = 6;  // Philox tags of the leverage-score draws
constexpr int kTagLevCols = 7;

// The launch sequence of one sketch on one stream.
cabs_status sketch_enqueue(const cabs_source& src, const cabs_params& p, void* ws, size_t ws_bytes, cudaStream_t s,
                           const cabs_result& out, bool fork_sides) {
  Carve cv(ws, ws_bytes);
  SketchWs w = carve_sketch(cv, src, p);
  if (!cv.fits()) {
    set_error("sketch workspace too small: need %zu bytes, got %zu", cv.used, ws_bytes);
    return CABS_ENOMEM;
  }
  const bool f64 = p.prec == CABS_PREC_FP64;
  const int64_t m = p.m, n = p.n;
  const int k1 = p.k1, k2 = p.k2;
  cabs_diag* dg = out.diag ? out.diag : w.diag;
  CABS_LAUNCH(s, "diag_clear_kernel", diag_clear_kernel<<<1, 256, 0, s>>>(dg));
  // Algorithm 2, step 1: pilot sampling
  CABS_TRY(launch_draw2(p.seed, 0, m, k1, w.pr_drawn, out.pilot_rows, 1, n, k1, w.pc_drawn, out.pilot_cols, s));
  CABS_TRY(launch_gather(src, m, n, out.pilot_rows, k1, out.pilot_cols, k1, f64, w.C, w.Rt, w.W, s));
  // step 2: pilot sketching and embeddings P, Q
  CABS_TRY(launch_core(m, n, k1, f64, tc_extrap_ok(p.prec), p.core, p.trunc_rtol, w.C, w.Rt, w.W, true, w.P, w.S_pilot, w.Q,
                       &dg->rank_pilot, &dg->sweeps_pilot, &dg->refine_pilot, &dg->status, nullptr, nullptr, nullptr, w.core,
                       w.core_bytes, s));
  if (p.flags & CABS_FLAG_HARD_THRESHOLD) {
    // step 3, hard-threshold variant (Section 5): largest-norm rows of P and Q
    CABS_TRY(launch_threshold(w.P, m, k1, k2, p.prec, out.rows, w.side_r, w.side_r_bytes, s));
    CABS_TRY(launch_threshold(w.Q, n, k1, k2, p.prec, out.cols, w.side_c, w.side_c_bytes, s));
  } else if (p.flags & CABS_FLAG_LEVERAGE) {
    // step 3, leverage-score variant (Section 5): P Q^T in SVD form
    // (supplementary Section 3), its leverage scores as sampling probabilities
    CABS_LAUNCH(s, "fill_kernel", fill_kernel<<<1, 256, 0, s>>>(w.lev_one, k1, 1.0));
    CABS_TRY(launch_orthogonalize(m, n, k1, f64, p.trunc_rtol, w.P, w.lev_one, w.Q, w.lev_X, w.lev_s, w.lev_Y, nullptr,
                                  &dg->status, w.core, w.core_bytes, s));
    CABS_TRY(launch_leverage_select(w.lev_X, m, k1, k2, f64, p.seed, kTagLevRows, out.rows, w.side_r, w.side_r_bytes,
                                    s));
    CABS_TRY(launch_leverage_select(w.lev_Y, n, k1, k2, f64, p.seed, kTagLevCols, out.cols, w.side_c, w.side_c_bytes,
                                    s));
  } else {
    // step 3: weighted k-means on P and Q, snap to rows. The two sides are
    // independent (their own workspaces; the shared diagnostics are updated
    // atomically): for a sketch on its own the column side runs on the side
    // stream, forked after the pilot and joined before the follow-up gather
    // (in a batch it stays on the lane's stream: the lanes are concurrent
    // already, and more streams measured slower there).
    SideStream ss;
    ss.s = s;
    if (fork_sides) {
      CABS_TRY(side_stream_of(s, ss));
      if (cudaEventRecord(ss.fork, s) != cudaSuccess || cudaStreamWaitEvent(ss.s, ss.fork, 0) != cudaSuccess)
        return check_cuda("side stream fork");
    }
    CABS_TRY(launch_kmeans(w.Q, n, k1, w.pc_drawn, k2, p.iters, p.prec, p.upsilon_pow, nullptr, w.Zc, dg->e_cols,
                           &dg->T_cols, &dg->rechecked, w.side_c, w.side_c_bytes, ss.s));
    CABS_TRY(launch_snap(w.Q, n, k1, w.Zc, k2, p.prec, w.fc_order, out.cols, w.side_c, w.side_c_bytes,
                         &dg->snap_fallbacks, &dg->status, ss.s));
    if (p.flags & CABS_FLAG_FOLLOW_ERR)
      CABS_TRY(launch_encoding_error(w.Q, n, k1, out.cols, k2, p.prec, p.upsilon_pow, &dg->e_follow_cols, w.side_c,
                                     w.side_c_bytes, ss.s));
    CABS_TRY(launch_kmeans(w.P, m, k1, w.pr_drawn, k2, p.iters, p.prec, p.upsilon_pow, nullptr, w.Zr, dg->e_rows,
                           &dg->T_rows, &dg->rechecked, w.side_r, w.side_r_bytes, s));
    CABS_TRY(launch_snap(w.P, m, k1, w.Zr, k2, p.prec, w.fr_order, out.rows, w.side_r, w.side_r_bytes,
                         &dg->snap_fallbacks, &dg->status, s));
    if (p.flags & CABS_FLAG_FOLLOW_ERR)
      CABS_TRY(launch_encoding_error(w.P, m, k1, out.rows, k2, p.prec, p.upsilon_pow, &dg->e_follow_rows, w.side_r,
                                     w.side_r_bytes, s));
    if (fork_sides &&
        (cudaEventRecord(ss.join, ss.s) != cudaSuccess || cudaStreamWaitEvent(s, ss.join, 0) != cudaSuccess))
      return check_cuda("side stream join");
  }
  if ((p.flags & CABS_FLAG_FOLLOW_ERR) && (p.flags & (CABS_FLAG_HARD_THRESHOLD | CABS_FLAG_LEVERAGE))) {
    CABS_TRY(launch_encoding_error(w.P, m, k1, out.rows, k2, p.prec, p.upsilon_pow, &dg->e_follow_rows, w.side_r,
                                   w.side_r_bytes, s));
    CABS_TRY(launch_encoding_error(w.Q, n, k1, out.cols, k2, p.prec, p.upsilon_pow, &dg->e_follow_cols, w.side_c,
                                   w.side_c_bytes, s));
  }
  // steps 3-4: follow-up gather and sketching
  CABS_TRY(launch_gather(src, m, n, out.rows, k2, out.cols, k2, f64, w.C, w.Rt, w.W, s));
  const bool svd_form = (p.flags & CABS_FLAG_SVD_FORM) != 0;
  // with the SVD form, the factors go to the (now free) embedding buffers first
  void* U1 = svd_form ? w.P : out.U;
  void* V1 = svd_form ? w.Q : out.V;
  double* S1 = svd_form ? w.S_pilot : out.S;
  CABS_TRY(launch_core(m, n, k2, f64, tc_extrap_ok(p.prec), p.core, p.trunc_rtol, w.C, w.Rt, w.W, false, U1, S1, V1, &dg->rank_final,
                       &dg->sweeps_final, &dg->refine_final, &dg->status, nullptr, nullptr, nullptr, w.core,
                       w.core_bytes, s));
  // supplementary Section 3: orthogonalisation into SVD form
  if (svd_form)
    CABS_TRY(launch_orthogonalize(m, n, k2, f64, p.trunc_rtol, U1, S1, V1, out.U, out.S, out.V, &dg->rank_final,
                                  &dg->status, w.core, w.core_bytes, s));
  // Section 5: relative Frobenius error of the result
  if (p.flags & CABS_FLAG_ERROR) {
    CABS_TRY(launch_error(src, m, n, k2, f64, p.prec, out.U, out.S, out.V, p.err_samples, p.err_seed, w.err_ws,
                          w.err_bytes, w.err_out2, s));
    CABS_LAUNCH(s, "err_finalize_kernel", err_finalize_kernel<<<1, 32, 0, s>>>(w.err_out2, out.err));
  }
  return CABS_OK;
}

cabs_status validate_result(const cabs_result* out) {
  CABS_REQUIRE(out != nullptr, "result is NULL");
  CABS_REQUIRE(out->U && out->S && out->V, "result: U, S and V must be set");
  CABS_REQUIRE(out->rows && out->cols && out->pilot_rows && out->pilot_cols, "result: index buffers must be set");
  return CABS_OK;
}

}  // namespace cabs

using namespace cabs;

extern "C" {

const char* cabs_version(void) { return "libcabs 0.1 (sm_103a)"; }

const char* cabs_last_error(cabs_ctx*) { return last_error(); }

cabs_status cabs_create(cabs_ctx** out, int device) {
  clear_error();
  CABS_REQUIRE(out != nullptr, "out is NULL");
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count <= 0) {
    cudaGetLastError();
    set_error("no CUDA device available");
    return CABS_ECUDA;
  }
  CABS_REQUIRE(device >= 0 && device < count, "device %d outside [0, %d)", device, count);
  DeviceGuard g(device);
  if (!g.ok) {
    set_error("cannot select CUDA device %d", device);
    return CABS_ECUDA;
  }
  cabs_ctx* c = new cabs_ctx();
  c->device = device;
  if (cudaEventCreateWithFlags(&c->fork_event, cudaEventDisableTiming) != cudaSuccess) {
    delete c;
    return check_cuda("cudaEventCreate");
  }
  *out = c;
  return CABS_OK;
}

void cabs_destroy(cabs_ctx* ctx) {
  if (!ctx) return;
  cabs_serve_stop(ctx);
  DeviceGuard g(ctx->device);
  for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
  for (cudaStream_t s : ctx->lanes) cudaStreamDestroy(s);
  for (cudaEvent_t e : ctx->lane_events) cudaEventDestroy(e);
  if (ctx->fork_event) cudaEventDestroy(ctx->fork_event);
  delete ctx;
}

cabs_status cabs_set_wait_limit(cabs_ctx* ctx, int64_t polls) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  g_wait_limit.store(polls < 0 ? (long long)CABS_WAIT_LIMIT_DEFAULT : (long long)polls, std::memory_order_relaxed);
  return CABS_OK;
}

cabs_status cabs_workspace_size(const cabs_source* src, const cabs_params* p, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_TRY(validate_params(p));
  CABS_TRY(validate_source(src, p->m, p->n));
  *bytes = sketch_ws_bytes(*src, *p);
  return CABS_OK;
}

cabs_status cabs_sketch(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p, void* ws, size_t ws_bytes,
                        cabs_stream stream, const cabs_result* out) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_TRY(validate_params(p));
  CABS_TRY(validate_source(src, p->m, p->n));
  CABS_TRY(validate_result(out));
  CABS_TRY(validate_error_request(src, p, out));
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  const size_t need = sketch_ws_bytes(*src, *p);
  if (ws_bytes < need) {
    set_error("workspace too small: need %zu bytes, got %zu", need, ws_bytes);
    return CABS_ENOMEM;
  }
  DeviceGuard g(ctx->device);
  if (!g.ok) {
    set_error("cannot select CUDA device %d", ctx->device);
    return CABS_ECUDA;
  }
  TuneScope shape(tune_lookup(ctx, *p));
  return sketch_enqueue(*src, *p, ws, ws_bytes, (cudaStream_t)stream, *out);
}

cabs_status cabs_error_workspace_size(const cabs_source* src, const cabs_params* p, int64_t samples, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_TRY(validate_params(p));
  CABS_TRY(validate_source(src, p->m, p->n));
  CABS_REQUIRE(samples >= 0, "samples must be >= 0");
  CABS_REQUIRE(samples > 0 || src->kind != CABS_SRC_RBF, "the exact error needs stored entries (dense or CSR)");
  *bytes = error_ws_bytes(*src, p->m, p->n, p->k2, samples, p->prec) + 256;
  return CABS_OK;
}

cabs_status cabs_error(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p, const cabs_result* res,
                       int64_t samples, uint64_t seed, void* ws, size_t ws_bytes, cabs_stream stream,
                       double* rel_fro) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && rel_fro != nullptr, "ctx and rel_fro must be non-NULL");
  CABS_TRY(validate_params(p));
  CABS_TRY(validate_source(src, p->m, p->n));
  CABS_REQUIRE(res != nullptr && res->U && res->S && res->V, "result U, S, V must be set");
  size_t need = 0;
  CABS_TRY(cabs_error_workspace_size(src, p, samples, &need));
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  if (ws_bytes < need) {
    set_error("error workspace too small: need %zu bytes, got %zu", need, ws_bytes);
    return CABS_ENOMEM;
  }
  DeviceGuard g(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  double* out2 = (double*)ws;
  void* part = (char*)ws + 256;
  CABS_TRY(launch_error(*src, p->m, p->n, p->k2, p->prec == CABS_PREC_FP64, p->prec, res->U, res->S, res->V, samples,
                        seed, part, ws_bytes - 256, out2, s));
  double h[2] = {0.0, 0.0};
  if (cudaMemcpyAsync(h, out2, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return check_cuda("cabs_error readback");
  *rel_fro = h[1] > 0.0 ? std::sqrt(h[0] / h[1]) : 0.0;
  return CABS_OK;
}

// ------------------------------------------------------------ step calls

cabs_status cabs_draw_indices(cabs_ctx* ctx, uint64_t seed, int32_t tag, int64_t N, int32_t k, int32_t* d_drawn,
                              int32_t* d_sorted, cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(N >= 1 && N < (int64_t)INT32_MAX, "N outside [1, 2^31)");
  CABS_REQUIRE(k >= 0 && k <= N && k <= 4096, "k outside [0, min(N, 4096)]");
  CABS_REQUIRE(k == 0 || (d_drawn && d_sorted), "output buffers are NULL");
  if (k == 0) return CABS_OK;
  DeviceGuard g(ctx->device);
  return launch_draw2(seed, tag, N, k, d_drawn, d_sorted, 0, 1, 0, nullptr, nullptr, (cudaStream_t)stream);
}

cabs_status cabs_gather(cabs_ctx* ctx, const cabs_source* src, int64_t m, int64_t n, const int32_t* d_rows,
                        int32_t k_r, const int32_t* d_cols, int32_t k_c, int32_t prec, void* C, void* Rt, double* W,
                        cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(m >= 1 && n >= 1 && m < INT32_MAX && n < INT32_MAX, "m, n outside [1, 2^31)");
  CABS_TRY(validate_source(src, m, n));
  CABS_REQUIRE(k_r >= 0 && k_r <= CABS_MAX_K && k_c >= 0 && k_c <= CABS_MAX_K, "k_r, k_c outside [0, %d]",
               CABS_MAX_K);
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  CABS_REQUIRE(!C || k_c == 0 || d_cols, "cols is NULL");
  CABS_REQUIRE(!Rt || k_r == 0 || d_rows, "rows is NULL");
  CABS_REQUIRE(!W || (C && d_rows), "W needs C and rows");
  DeviceGuard g(ctx->device);
  return launch_gather(*src, m, n, d_rows, k_r, d_cols, k_c, prec == CABS_PREC_FP64, C, Rt, W, (cudaStream_t)stream);
}

cabs_status cabs_sketching_workspace_size(int64_t m, int64_t n, int32_t k, int32_t prec, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_REQUIRE(m >= 1 && n >= 1 && k >= 1 && k <= CABS_MAX_K && k <= std::min(m, n), "bad m, n, k");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  *bytes = core_ws_bytes(m, n, k, prec == CABS_PREC_FP64);
  return CABS_OK;
}

cabs_status cabs_sketching(cabs_ctx* ctx, int64_t m, int64_t n, int32_t k, int32_t prec, int32_t core, double trunc_rtol,
                      const void* C, const void* Rt, const double* W, int32_t embed, void* out1, double* S,
                      void* out2, int32_t* d_rank, int32_t* d_sweeps, double* d_sig, double* d_Uw, double* d_Vw,
                      void* ws, size_t ws_bytes, cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(m >= 1 && n >= 1 && k >= 1 && k <= CABS_MAX_K && k <= std::min(m, n), "bad m, n, k");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  CABS_REQUIRE(core == CABS_CORE_PINV || core == CABS_CORE_STABILIZED, "unknown core");
  CABS_REQUIRE(C && Rt && W && out1 && S && out2, "NULL input or output");
  CABS_REQUIRE(std::isfinite(trunc_rtol) && trunc_rtol >= 0.0, "bad trunc_rtol");
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  DeviceGuard g(ctx->device);
  return launch_core(m, n, k, prec == CABS_PREC_FP64, tc_extrap_ok(prec), core, trunc_rtol, C, Rt, W, embed != 0, out1, S, out2, d_rank,
                     d_sweeps, nullptr, nullptr, d_sig, d_Uw, d_Vw, ws, ws_bytes, (cudaStream_t)stream);
}

cabs_status cabs_kmeans_workspace_size(int64_t M, int32_t d, int32_t k2, int32_t iters, int32_t prec, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_REQUIRE(M >= 1 && M < INT32_MAX && d >= 1 && d <= CABS_MAX_K && k2 >= 1 && k2 <= CABS_MAX_K && k2 <= M,
               "bad M, d, k2");
  CABS_REQUIRE(iters >= 0 && iters <= CABS_MAX_ITERS, "bad iters");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  *bytes = kmeans_ws_bytes(M, d, k2, iters, prec);
  return CABS_OK;
}

cabs_status cabs_kmeans(cabs_ctx* ctx, const void* X, int64_t M, int32_t d, const int32_t* d_init_rows, int32_t k2,
                        int32_t iters, int32_t prec, float upsilon_pow, int32_t* d_labels, void* d_centres,
                        double* d_energy, int32_t* d_T, void* ws, size_t ws_bytes, cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(M >= 1 && M < INT32_MAX && d >= 1 && d <= CABS_MAX_K && k2 >= 1 && k2 <= CABS_MAX_K && k2 <= M,
               "bad M, d, k2");
  CABS_REQUIRE(iters >= 0 && iters <= CABS_MAX_ITERS, "bad iters");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  CABS_REQUIRE(X && d_init_rows && d_centres, "NULL input or output");
  CABS_REQUIRE(std::isfinite(upsilon_pow), "upsilon_pow must be finite");
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  DeviceGuard g(ctx->device);
  return launch_kmeans(X, M, d, d_init_rows, k2, iters, prec, upsilon_pow, d_labels, d_centres, d_energy, d_T, nullptr,
                       ws, ws_bytes, (cudaStream_t)stream);
}

cabs_status cabs_snap_workspace_size(int64_t M, int32_t d, int32_t k2, int32_t prec, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_REQUIRE(M >= 1 && M < INT32_MAX && d >= 1 && d <= CABS_MAX_K && k2 >= 1 && k2 <= CABS_MAX_K && k2 <= M,
               "bad M, d, k2");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  *bytes = snap_ws_bytes(M, d, k2, prec);
  return CABS_OK;
}

cabs_status cabs_snap(cabs_ctx* ctx, const void* X, int64_t M, int32_t d, const void* Z, int32_t k2, int32_t prec,
                      int32_t* d_order, int32_t* d_sorted, void* ws, size_t ws_bytes, cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(M >= 1 && M < INT32_MAX && d >= 1 && d <= CABS_MAX_K && k2 >= 1 && k2 <= CABS_MAX_K && k2 <= M,
               "bad M, d, k2");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  CABS_REQUIRE(X && Z && d_order && d_sorted, "NULL input or output");
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  DeviceGuard g(ctx->device);
  return launch_snap(X, M, d, Z, k2, prec, d_order, d_sorted, ws, ws_bytes, nullptr, nullptr, (cudaStream_t)stream);
}

cabs_status cabs_threshold_workspace_size(int64_t M, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_REQUIRE(M >= 1 && M < INT32_MAX, "M outside [1, 2^31)");
  *bytes = threshold_ws_bytes(M);
  return CABS_OK;
}

cabs_status cabs_threshold(cabs_ctx* ctx, const void* X, int64_t M, int32_t d, int32_t k2, int32_t prec,
                           int32_t* d_sorted, void* ws, size_t ws_bytes, cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(M >= 1 && M < INT32_MAX && d >= 1 && k2 >= 1 && k2 <= M, "bad M, d, k2");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  CABS_REQUIRE(X && d_sorted, "NULL input or output");
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  DeviceGuard g(ctx->device);
  return launch_threshold(X, M, d, k2, prec, d_sorted, ws, ws_bytes, (cudaStream_t)stream);
}

cabs_status cabs_orthogonalize_workspace_size(int64_t m, int64_t n, int32_t k, int32_t prec, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_REQUIRE(m >= 1 && n >= 1 && k >= 1 && k <= CABS_MAX_K, "bad m, n, k");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  *bytes = orth_ws_bytes(m, n, k, prec == CABS_PREC_FP64);
  return CABS_OK;
}

static bool overlaps(const void* a, size_t na, const void* b, size_t nb) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  return x < y + nb && y < x + na;
}

cabs_status cabs_orthogonalize(cabs_ctx* ctx, int64_t m, int64_t n, int32_t k, int32_t prec, double trunc_rtol,
                               const void* U, const double* S, const void* V, void* X, double* s, void* Y,
                               int32_t* d_rank, void* ws, size_t ws_bytes, cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(m >= 1 && n >= 1 && k >= 1 && k <= CABS_MAX_K, "bad m, n, k");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "unknown precision");
  CABS_REQUIRE(U && S && V && X && s && Y, "NULL input or output");
  CABS_REQUIRE(std::isfinite(trunc_rtol) && trunc_rtol >= 0.0, "bad trunc_rtol");
  const size_t e = prec == CABS_PREC_FP64 ? 8 : 4;
  const size_t bu = (size_t)m * k * e, bv = (size_t)n * k * e;
  CABS_REQUIRE(!overlaps(X, bu, U, bu) && !overlaps(X, bu, V, bv) && !overlaps(Y, bv, U, bu) &&
                   !overlaps(Y, bv, V, bv) && !overlaps(X, bu, Y, bv),
               "X and Y must not overlap U, V or each other");
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  DeviceGuard g(ctx->device);
  return launch_orthogonalize(m, n, k, prec == CABS_PREC_FP64, trunc_rtol, U, S, V, X, s, Y, d_rank, nullptr, ws,
                              ws_bytes, (cudaStream_t)stream);
}

static cabs_status validate_cur(const cabs_source* src, const cabs_cur_params* p) {
  CABS_REQUIRE(src != nullptr && p != nullptr, "NULL source or params");
  CABS_REQUIRE(p->m >= 1 && p->n >= 1 && p->m < (int64_t)INT32_MAX && p->n < (int64_t)INT32_MAX, "bad m, n");
  const int64_t mn = std::min<int64_t>({p->m, p->n, (int64_t)CABS_MAX_K});
  CABS_REQUIRE(p->kb >= 1 && p->kb <= mn && p->kt >= 1 && p->kt <= mn, "kb = %d, kt = %d outside [1, min(m, n, %d)]",
               p->kb, p->kt, CABS_MAX_K);
  CABS_REQUIRE(p->prec >= CABS_PREC_FP64 && p->prec <= CABS_PREC_BF16, "unknown precision %d", p->prec);
  CABS_REQUIRE(std::isfinite(p->trunc_rtol) && p->trunc_rtol >= 0.0, "trunc_rtol must be finite and >= 0");
  return validate_source(src, p->m, p->n);
}

cabs_status cabs_sketch_cur_workspace_size(const cabs_source* src, const cabs_cur_params* p, size_t* bytes) {
  clear_error();
  CABS_REQUIRE(bytes != nullptr, "bytes is NULL");
  CABS_TRY(validate_cur(src, p));
  *bytes = cur_ws_bytes(p->m, p->n, p->kb, p->kt, p->prec == CABS_PREC_FP64);
  return CABS_OK;
}

cabs_status cabs_sketch_cur(cabs_ctx* ctx, const cabs_source* src, const cabs_cur_params* p, void* ws,
                            size_t ws_bytes, cabs_stream stream, const cabs_cur_result* out) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_TRY(validate_cur(src, p));
  CABS_REQUIRE(out && out->U && out->S && out->V && out->rows_b && out->cols_b && out->rows_t && out->cols_t,
               "NULL output");
  CABS_REQUIRE(ws != nullptr && ((uintptr_t)ws & 255) == 0, "workspace must be non-NULL and 256-byte aligned");
  DeviceGuard g(ctx->device);
  return launch_sketch_cur(*src, p->m, p->n, p->kb, p->kt, p->seed, p->prec == CABS_PREC_FP64, p->trunc_rtol, out->U,
                           out->S, out->V, out->Ustar, out->rows_b, out->cols_b, out->rows_t, out->cols_t, out->ranks,
                           ws, ws_bytes, (cudaStream_t)stream);
}

}  // extern "C"

// ---------------------------------------------------------------- batched

namespace cabs {

static uint64_t mix(uint64_t h, uint64_t v) {
  h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
  return h;
}

static uint64_t batch_key(int count, const cabs_source* src, const cabs_params* p, void* ws, const size_t* off,
                          const cabs_result* out, int lanes) {
  uint64_t h = mix(0, (uint64_t)count);
  h = mix(h, (uint64_t)(uintptr_t)ws);
  h = mix(h, (uint64_t)lanes);
  for (int i = 0; i < count; ++i) {
    const uint64_t* a = (const uint64_t*)&src[i];
    for (size_t j = 0; j < sizeof(cabs_source) / 8; ++j) h = mix(h, a[j]);
    const uint64_t* b = (const uint64_t*)&p[i];
    for (size_t j = 0; j < sizeof(cabs_params) / 8; ++j) h = mix(h, b[j]);
    const uint64_t* c = (const uint64_t*)&out[i];
    for (size_t j = 0; j < sizeof(cabs_result) / 8; ++j) h = mix(h, c[j]);
    h = mix(h, (uint64_t)off[i]);
  }
  return h;
}

cabs_status ensure_lanes(cabs_ctx* ctx, int lanes) {
  while ((int)ctx->lanes.size() < lanes) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return check_cuda("cudaStreamCreate");
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return check_cuda("cudaEventCreate");
    ctx->lanes.push_back(s);
    ctx->lane_events.push_back(e);
  }
  return CABS_OK;
}

cabs_status batched_enqueue(cabs_ctx* ctx, int count, const cabs_source* src, const cabs_params* p, void* ws,
                                   const size_t* off, const cabs_result* out, int lanes, cudaStream_t s) {
  // largest members first, dealt round-robin to the lanes
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const double wa = (double)(p[a].m + p[a].n) * p[a].k1 * p[a].k1;
    const double wb = (double)(p[b].m + p[b].n) * p[b].k1 * p[b].k1;
    return wa > wb;
  });
  if (cudaEventRecord(ctx->fork_event, s) != cudaSuccess) return check_cuda("fork record");
  for (int l = 0; l < lanes; ++l)
    if (cudaStreamWaitEvent(ctx->lanes[l], ctx->fork_event, 0) != cudaSuccess) return check_cuda("fork wait");
  SharersScope sharing(std::min(lanes, count));
  for (int t = 0; t < count; ++t) {
    const int i = order[t];
    const size_t need = sketch_ws_bytes(src[i], p[i]);
    TuneScope shape(tune_lookup(ctx, p[i]));
    CABS_TRY(sketch_enqueue(src[i], p[i], (char*)ws + off[i], need, ctx->lanes[t % lanes], out[i], false));
  }
  for (int l = 0; l < lanes; ++l) {
    if (cudaEventRecord(ctx->lane_events[l], ctx->lanes[l]) != cudaSuccess) return check_cuda("join record");
    if (cudaStreamWaitEvent(s, ctx->lane_events[l], 0) != cudaSuccess) return check_cuda("join wait");
  }
  return CABS_OK;
}

}  // namespace cabs

extern "C" cabs_status cabs_sketch_batched(cabs_ctx* ctx, int32_t count, const cabs_source* src, const cabs_params* p,
                                           void* ws, const size_t* ws_offsets, const cabs_result* out, int32_t lanes,
                                           int32_t use_graph, cabs_stream stream) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(count >= 0, "count < 0");
  if (count == 0) return CABS_OK;
  CABS_REQUIRE(src && p && out && ws && ws_offsets, "NULL array");
  CABS_REQUIRE(lanes >= 0 && lanes <= 16, "lanes outside [0, 16]");
  if (lanes == 0) {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    lanes = ctx->tuned_lanes > 0 ? ctx->tuned_lanes : 8;
  }
  for (int i = 0; i < count; ++i) {
    CABS_TRY(validate_params(&p[i]));
    CABS_TRY(validate_source(&src[i], p[i].m, p[i].n));
    CABS_TRY(validate_result(&out[i]));
    CABS_TRY(validate_error_request(&src[i], &p[i], &out[i]));
    CABS_REQUIRE((ws_offsets[i] & 255) == 0, "member %d: workspace offset not 256-aligned", i);
  }
  DeviceGuard g(ctx->device);
  CABS_TRY(ensure_lanes(ctx, lanes));
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) return batched_enqueue(ctx, count, src, p, ws, ws_offsets, out, lanes, s);
  CABS_REQUIRE(s != nullptr, "graph replay needs a non-default stream");
  uint64_t key = batch_key(count, src, p, ws, ws_offsets, out, lanes);
  {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    key = mix(key, ctx->tune_version);  // launch shapes changed: capture again
  }
  std::lock_guard<std::mutex> lock(ctx->graph_mu);
  auto it = ctx->graphs.find(key);
  if (it == ctx->graphs.end()) {
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return check_cuda("cudaStreamBeginCapture");
    const long long l0 = thread_launches();
    const cabs_status st = batched_enqueue(ctx, count, src, p, ws, ws_offsets, out, lanes, s);
    const long long captured = thread_launches() - l0;
    add_launches(-captured);  // captured, not run; counted again at every replay
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (st != CABS_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (ce != cudaSuccess) return check_cuda("cudaStreamEndCapture");
    GraphEntry ge;
    ge.launches = captured;
    const cudaError_t ie = cudaGraphInstantiate(&ge.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return check_cuda("cudaGraphInstantiate");
    if (ctx->graphs.size() >= 32) {
      for (auto& kv : ctx->graphs) cudaGraphExecDestroy(kv.second.exec);
      ctx->graphs.clear();
    }
    it = ctx->graphs.emplace(key, ge).first;
  }
  if (cudaGraphLaunch(it->second.exec, s) != cudaSuccess) return check_cuda("cudaGraphLaunch");
  add_launches(it->second.launches);
  return CABS_OK;
}
