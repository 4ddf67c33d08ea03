// Launch-shape tuning: the per-context table of cabs_tune entries by shape
// bucket, its cache file, and the autotuner that fills it from timed trials.
//
// A bucket is (prec, ceil(k2 / 32), floor(log2(m + n))): the knobs change the
// work split of kernels whose cost grows with the embedding width (the
// extrapolation GEMMs and the tensor-core assignment: output columns per
// thread and per column block) and with the number of rows (the column
// gather: rows in flight per warp). None of them changes a result, so the
// autotuner may pick any candidate; it keeps the fastest.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include "api_internal.cuh"
#include "common.cuh"
#include "profile.cuh"

namespace cabs {

namespace {
thread_local cabs_tune t_tune = {0, 0, 0, 0};

bool tune_valid(const cabs_tune& t) {
  const bool tn = t.extrap_tn == 0 || t.extrap_tn == 2 || t.extrap_tn == 4 || t.extrap_tn == 8;
  const bool gr = t.gather_rows == 0 || t.gather_rows == 2 || t.gather_rows == 4 || t.gather_rows == 8;
  const bool bn = t.assign_bn == 0 || t.assign_bn == 128 || t.assign_bn == 256;
  return tn && gr && bn && t.reserved == 0;
}

int size_bucket(int64_t m, int64_t n) {
  const double s = (double)std::max<int64_t>(m + n, 1);
  return std::min(63, (int)std::floor(std::log2(s)));
}
}  // namespace

const cabs_tune& current_tune() { return t_tune; }

TuneScope::TuneScope(const cabs_tune& t) : prev(t_tune) { t_tune = t; }
TuneScope::~TuneScope() { t_tune = prev; }

uint32_t tune_bucket(int prec, int k, int64_t m, int64_t n) {
  const uint32_t kb = (uint32_t)std::min(255, (std::max(k, 1) + 31) / 32);
  return ((uint32_t)(prec & 0xff) << 16) | (kb << 8) | (uint32_t)size_bucket(m, n);
}

cabs_tune tune_lookup(cabs_ctx* ctx, const cabs_params& p) {
  cabs_tune t = {0, 0, 0, 0};
  if (!ctx) return t;
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  auto it = ctx->tune.find(tune_bucket(p.prec, p.k2, p.m, p.n));
  if (it != ctx->tune.end()) t = it->second;
  return t;
}

}  // namespace cabs

using namespace cabs;

extern "C" cabs_status cabs_tune_set(cabs_ctx* ctx, int32_t prec, int32_t k2, int64_t m, int64_t n,
                                     const cabs_tune* t) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(prec >= CABS_PREC_FP64 && prec <= CABS_PREC_BF16, "prec %d unknown", prec);
  CABS_REQUIRE(k2 >= 1 && k2 <= CABS_MAX_K && m >= 1 && n >= 1, "k2, m, n out of range");
  if (t) {
    CABS_REQUIRE(tune_valid(*t), "cabs_tune: extrap_tn in {0,2,4,8}, gather_rows in {0,2,4,8}, "
                                 "assign_bn in {0,128,256}, reserved 0");
    CABS_REQUIRE(!(prec == CABS_PREC_FP64 && t->extrap_tn == 8), "extrap_tn 8 is for the FP32 modes only");
  }
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  const uint32_t b = tune_bucket(prec, k2, m, n);
  if (t)
    ctx->tune[b] = *t;
  else
    ctx->tune.erase(b);
  ++ctx->tune_version;
  return CABS_OK;
}

extern "C" cabs_status cabs_tune_get(cabs_ctx* ctx, int32_t prec, int32_t k2, int64_t m, int64_t n, cabs_tune* t,
                                     int32_t* found) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && t != nullptr, "ctx and t must be non-NULL");
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  auto it = ctx->tune.find(tune_bucket(prec, k2, m, n));
  *t = it != ctx->tune.end() ? it->second : cabs_tune{0, 0, 0, 0};
  if (found) *found = it != ctx->tune.end() ? 1 : 0;
  return CABS_OK;
}

extern "C" cabs_status cabs_tune_save(cabs_ctx* ctx, const char* path) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && path != nullptr, "ctx and path must be non-NULL");
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  FILE* f = std::fopen(path, "w");
  CABS_REQUIRE(f != nullptr, "cannot write %s", path);
  std::fprintf(f, "# libcabs launch shapes: bucket prec kb sb extrap_tn gather_rows assign_bn\n");
  std::vector<uint32_t> keys;
  for (auto& kv : ctx->tune) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end());
  for (uint32_t b : keys) {
    const cabs_tune& t = ctx->tune[b];
    std::fprintf(f, "bucket %u %u %u %d %d %d\n", b >> 16, (b >> 8) & 0xff, b & 0xff, t.extrap_tn, t.gather_rows,
                 t.assign_bn);
  }
  std::fprintf(f, "lanes %d\n", ctx->tuned_lanes);
  const bool ok = std::fclose(f) == 0;
  CABS_REQUIRE(ok, "cannot finish writing %s", path);
  return CABS_OK;
}

extern "C" cabs_status cabs_tune_load(cabs_ctx* ctx, const char* path) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && path != nullptr, "ctx and path must be non-NULL");
  FILE* f = std::fopen(path, "r");
  CABS_REQUIRE(f != nullptr, "cannot read %s", path);
  std::unordered_map<uint32_t, cabs_tune> table;
  int lanes = 0;
  char line[256];
  int lineno = 0;
  bool bad = false;
  while (!bad && std::fgets(line, sizeof line, f)) {
    ++lineno;
    if (line[0] == '#' || line[0] == '\n') continue;
    unsigned pr, kb, sb;
    cabs_tune t = {0, 0, 0, 0};
    int l = 0;
    if (std::sscanf(line, "bucket %u %u %u %d %d %d", &pr, &kb, &sb, &t.extrap_tn, &t.gather_rows, &t.assign_bn) ==
        6) {
      bad = pr > CABS_PREC_BF16 || kb < 1 || kb > 255 || sb > 63 || !tune_valid(t);
      if (!bad) table[(pr << 16) | (kb << 8) | sb] = t;
    } else if (std::sscanf(line, "lanes %d", &l) == 1) {
      bad = l < 0 || l > 16;
      lanes = l;
    } else {
      bad = true;
    }
  }
  std::fclose(f);
  CABS_REQUIRE(!bad, "%s:%d: malformed launch-shape line", path, lineno);
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  ctx->tune.swap(table);
  ctx->tuned_lanes = lanes;
  ++ctx->tune_version;
  return CABS_OK;
}

// ------------------------------------------------------------- autotuner

namespace cabs {
namespace {

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  Timer() {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// Fastest of `reps` runs of one member's sketch under launch shape t (after
// one untimed run), in ms; < 0 on failure.
double time_member(const cabs_source& src, const cabs_params& p, void* ws, const cabs_result& out, const cabs_tune& t,
                   cudaStream_t s, Timer& tm, int reps) {
  TuneScope ts(t);
  SharersScope alone(1);
  const size_t need = sketch_ws_bytes(src, p);
  if (sketch_enqueue(src, p, ws, need, s, out, false) != CABS_OK) return -1.0;
  double best = 1e300;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(tm.a, s);
    if (sketch_enqueue(src, p, ws, need, s, out, false) != CABS_OK) return -1.0;
    cudaEventRecord(tm.b, s);
    if (cudaEventSynchronize(tm.b) != cudaSuccess) return -1.0;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, tm.a, tm.b);
    best = std::min(best, (double)ms);
  }
  return best;
}

}  // namespace
}  // namespace cabs

extern "C" cabs_status cabs_autotune(cabs_ctx* ctx, int32_t count, const cabs_source* src, const cabs_params* p,
                                     void* ws, const size_t* ws_offsets, const cabs_result* out, cabs_stream stream,
                                     int32_t* lanes_out) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(count >= 1, "count < 1");
  CABS_REQUIRE(src && p && out && ws && ws_offsets, "NULL array");
  for (int i = 0; i < count; ++i) {
    CABS_TRY(validate_params(&p[i]));
    CABS_TRY(validate_source(&src[i], p[i].m, p[i].n));
    CABS_TRY(validate_result(&out[i]));
    CABS_TRY(validate_error_request(&src[i], &p[i], &out[i]));
    CABS_REQUIRE((ws_offsets[i] & 255) == 0, "member %d: workspace offset not 256-aligned", i);
  }
  DeviceGuard g(ctx->device);
  if (!g.ok) {
    set_error("cannot select CUDA device %d", ctx->device);
    return CABS_ECUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Timer tm;
  CABS_REQUIRE(tm.a && tm.b, "cannot create CUDA events");
  // members by bucket; the representative is the member of median m + n
  std::unordered_map<uint32_t, std::vector<int>> groups;
  for (int i = 0; i < count; ++i) groups[tune_bucket(p[i].prec, p[i].k2, p[i].m, p[i].n)].push_back(i);
  std::vector<uint32_t> keys;
  for (auto& kv : groups) keys.push_back(kv.first);
  std::sort(keys.begin(), keys.end());
  constexpr int kReps = 5;
  for (uint32_t b : keys) {
    std::vector<int>& mem = groups[b];
    std::sort(mem.begin(), mem.end(), [&](int x, int y) { return p[x].m + p[x].n < p[y].m + p[y].n; });
    const int i = mem[mem.size() / 2];
    void* wsi = (char*)ws + ws_offsets[i];
    cabs_tune best = {0, 0, 0, 0};
    double tb = time_member(src[i], p[i], wsi, out[i], best, s, tm, kReps);
    if (tb < 0) return check_cuda("cabs_autotune: timing run");
    const bool f64 = p[i].prec == CABS_PREC_FP64;
    const bool tc = p[i].prec == CABS_PREC_TF32 || p[i].prec == CABS_PREC_BF16;
    std::vector<std::pair<int cabs_tune::*, std::vector<int>>> knobs;
    knobs.push_back({&cabs_tune::extrap_tn, f64 ? std::vector<int>{2, 4} : std::vector<int>{2, 4, 8}});
    if (src[i].kind == CABS_SRC_DENSE) knobs.push_back({&cabs_tune::gather_rows, {2, 4, 8}});
    if (tc) knobs.push_back({&cabs_tune::assign_bn, {128, 256}});
    for (auto& kn : knobs) {
      for (int v : kn.second) {
        cabs_tune t = best;
        t.*(kn.first) = v;
        const double tt = time_member(src[i], p[i], wsi, out[i], t, s, tm, kReps);
        if (tt < 0) return check_cuda("cabs_autotune: timing run");
        if (tt < 0.98 * tb) {
          best = t;
          tb = tt;
        }
      }
    }
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tune[b] = best;
    ++ctx->tune_version;
  }
  // lanes for the whole batch, with the table just filled
  int best_l = 8;
  double best_ms = 1e300;
  for (int L : {4, 8, 12, 16}) {
    CABS_TRY(ensure_lanes(ctx, L));
    double ms_l = 1e300;
    for (int r = 0; r < 2; ++r) {
      cudaEventRecord(tm.a, s);
      CABS_TRY(batched_enqueue(ctx, count, src, p, ws, ws_offsets, out, L, s));
      cudaEventRecord(tm.b, s);
      if (cudaEventSynchronize(tm.b) != cudaSuccess) return check_cuda("cabs_autotune: batch timing");
      float ms = 0.f;
      cudaEventElapsedTime(&ms, tm.a, tm.b);
      ms_l = std::min(ms_l, (double)ms);
    }
    if (ms_l < best_ms) {
      best_ms = ms_l;
      best_l = L;
    }
  }
  {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    ctx->tuned_lanes = best_l;
    ++ctx->tune_version;
  }
  if (lanes_out) *lanes_out = best_l;
  return CABS_OK;
}
