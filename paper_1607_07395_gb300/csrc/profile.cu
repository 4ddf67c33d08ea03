// Per-kernel timing and launch counting for libcabs.
//
// When enabled, every kernel launch site records a CUDA event pair around the
// launch on the launching stream; cabs_profile_read synchronises the events
// and reports, per kernel name, the number of launches and the summed device
// time. The launch counter is always on (a relaxed atomic increment); a
// captured graph adds the launches it holds each time it is replayed.
// Profiling is process-wide and is skipped while the launching stream is
// being captured into a CUDA graph.
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "profile.cuh"

namespace cabs {
namespace {

struct Pending {
  std::string name;
  cudaEvent_t a, b;
};

std::atomic<long long> g_launches{0};
thread_local long long t_launches = 0;
std::atomic<int> g_enabled{0};
std::mutex g_mu;
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_pool;
struct Acc {
  long long launches = 0;
  double ms = 0.0;
};
std::map<std::string, Acc> g_acc;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &st) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return st != cudaStreamCaptureStatusNone;
}

void drain_locked() {
  for (auto& p : g_pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      Acc& a = g_acc[p.name];
      a.launches += 1;
      a.ms += ms;
    } else {
      cudaGetLastError();
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_pending.clear();
}

}  // namespace

ProfScope::ProfScope(cudaStream_t s, const char* name) : stream_(s), name_(name), a_(nullptr) {
  if (!g_enabled.load(std::memory_order_relaxed) || capturing(s)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  a_ = get_event();
  if (a_) cudaEventRecord(a_, s);
}

ProfScope::~ProfScope() {
  if (!a_) return;
  std::lock_guard<std::mutex> lk(g_mu);
  cudaEvent_t b = get_event();
  if (!b) return;
  cudaEventRecord(b, stream_);
  g_pending.push_back({name_, a_, b});
  if (g_pending.size() > 4096) drain_locked();
}

cabs_status launched(const char* what) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  ++t_launches;
  return check_cuda(what);
}

long long thread_launches() { return t_launches; }

void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

}  // namespace cabs

extern "C" {

cabs_status cabs_profile_enable(cabs_ctx* ctx, int32_t on) {
  (void)ctx;
  cabs::g_enabled.store(on ? 1 : 0);
  return CABS_OK;
}

int32_t cabs_profile_read(cabs_ctx* ctx, char* names, int32_t name_len, int64_t* launches, double* total_ms,
                          int32_t max, int32_t reset) {
  (void)ctx;
  std::lock_guard<std::mutex> lk(cabs::g_mu);
  cabs::drain_locked();
  int32_t i = 0;
  for (auto& kv : cabs::g_acc) {
    if (i >= max) break;
    if (names && name_len > 0) {
      std::strncpy(names + (size_t)i * name_len, kv.first.c_str(), name_len - 1);
      names[(size_t)i * name_len + name_len - 1] = 0;
    }
    if (launches) launches[i] = kv.second.launches;
    if (total_ms) total_ms[i] = kv.second.ms;
    ++i;
  }
  if (reset) cabs::g_acc.clear();
  return i;
}

int64_t cabs_launch_count(void) { return cabs::g_launches.load(); }

}  // extern "C"
