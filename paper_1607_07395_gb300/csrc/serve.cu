// Continuous-batching request loop (the serving form of the sketch).
//
// Requests arrive through cabs_serve_submit from any thread. A scheduler
// thread admits them in arrival order whenever one of `max_slots` slots is
// free and the request's device footprint (workspace + resident results)
// fits in the unused part of the caller's HBM arena; each admitted request
// is enqueued on its slot's stream, so requests admitted while others run
// overlap on the device. A finished request gives back its workspace at once
// and keeps its results (U, S, V, indices, diagnostics) resident in the arena
// until cabs_serve_release. The launch sequence of a request is the same as
// cabs_sketch's, so a result does not depend on what else was running.
//
// The scheduler waits on the host only (cudaEventQuery polling with short
// sleeps); nothing on the device waits for another request.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>

#include "api_internal.cuh"
#include "kernels.cuh"

namespace cabs {

using Clock = std::chrono::steady_clock;

// First-fit allocator over [0, size) with 256-byte granularity.
class ArenaAlloc {
 public:
  void reset(size_t size) {
    free_.clear();
    if (size) free_[0] = size;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }

 private:
  std::map<size_t, size_t> free_;
  size_t used_ = 0;
};

enum class ReqState { Queued, Running, Done, Failed };

struct Request {
  uint64_t ticket = 0;
  cabs_source src{};
  cabs_params p{};
  ReqState state = ReqState::Queued;
  cabs_status status = CABS_OK;
  size_t res_off = 0, res_bytes = 0, ws_off = 0, ws_bytes = 0;
  cabs_result res{};
  cabs_tune tune{};  // launch shape of the request's bucket, taken at submission
  double dev_start_ms = -1.0, dev_end_ms = -1.0;  // device-side interval, ms since the loop's epoch
  int slot = -1;
  Clock::time_point t_submit, t_done;
};

struct ServeState {
  char* arena = nullptr;
  size_t arena_bytes = 0;
  int device = 0;
  ArenaAlloc alloc;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;       // end of the slot's request (timing event)
  std::vector<cudaEvent_t> start_events; // start of the slot's request
  cudaEvent_t epoch = nullptr;           // recorded when the loop starts
  std::vector<uint64_t> slot_ticket;  // 0 = free
  std::deque<uint64_t> queue;
  std::map<uint64_t, Request> reqs;
  uint64_t next_ticket = 1;
  bool stopping = false;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::thread thread;
};

static size_t result_bytes(const cabs_params& p) {
  const size_t eb = elem_bytes(p.prec);
  Carve cv;
  cv.take<char>((size_t)p.m * p.k2 * eb);
  cv.take<double>(p.k2);
  cv.take<char>((size_t)p.n * p.k2 * eb);
  cv.take<int>(p.k2);
  cv.take<int>(p.k2);
  cv.take<int>(p.k1);
  cv.take<int>(p.k1);
  cv.take<cabs_diag>(1);
  cv.take<double>(1);
  return cv.used;
}

static cabs_result result_at(char* base, const cabs_params& p) {
  const size_t eb = elem_bytes(p.prec);
  Carve cv(base, (size_t)-1);
  cabs_result r;
  r.U = cv.take<char>((size_t)p.m * p.k2 * eb);
  r.S = cv.take<double>(p.k2);
  r.V = cv.take<char>((size_t)p.n * p.k2 * eb);
  r.rows = cv.take<int>(p.k2);
  r.cols = cv.take<int>(p.k2);
  r.pilot_rows = cv.take<int>(p.k1);
  r.pilot_cols = cv.take<int>(p.k1);
  r.diag = cv.take<cabs_diag>(1);
  r.err = cv.take<double>(1);
  return r;
}

// Called with the lock held: retire finished requests, then admit in order.
static void schedule_once(ServeState* st) {
  for (size_t s = 0; s < st->streams.size(); ++s) {
    const uint64_t t = st->slot_ticket[s];
    if (!t) continue;
    const cudaError_t q = cudaEventQuery(st->events[s]);
    if (q == cudaErrorNotReady) continue;
    Request& r = st->reqs[t];
    r.t_done = Clock::now();
    if (q == cudaSuccess) {
      r.state = ReqState::Done;
      float a = 0.f, b = 0.f;
      if (cudaEventElapsedTime(&a, st->epoch, st->start_events[s]) == cudaSuccess &&
          cudaEventElapsedTime(&b, st->epoch, st->events[s]) == cudaSuccess) {
        r.dev_start_ms = a;
        r.dev_end_ms = b;
      } else {
        cudaGetLastError();
      }
    } else {
      cudaGetLastError();
      r.state = ReqState::Failed;
      r.status = CABS_ECUDA;
    }
    st->alloc.release(r.ws_off, r.ws_bytes);
    r.ws_bytes = 0;
    st->slot_ticket[s] = 0;
    st->cv_done.notify_all();
  }
  while (!st->queue.empty()) {
    int slot = -1;
    for (size_t s = 0; s < st->streams.size(); ++s)
      if (!st->slot_ticket[s]) {
        slot = (int)s;
        break;
      }
    if (slot < 0) return;
    Request& r = st->reqs[st->queue.front()];
    size_t roff = 0, woff = 0;
    if (!st->alloc.alloc(r.res_bytes, &roff)) return;
    if (!st->alloc.alloc(r.ws_bytes, &woff)) {
      st->alloc.release(roff, r.res_bytes);
      return;
    }
    st->queue.pop_front();
    r.res_off = roff;
    r.ws_off = woff;
    r.res = result_at(st->arena + roff, r.p);
    r.slot = slot;
    r.state = ReqState::Running;
    SharersScope sharing((int)st->streams.size());
    TuneScope shape(r.tune);
    cudaEventRecord(st->start_events[slot], st->streams[slot]);
    const cabs_status s = sketch_enqueue(r.src, r.p, st->arena + woff, r.ws_bytes, st->streams[slot], r.res);
    if (s != CABS_OK || cudaEventRecord(st->events[slot], st->streams[slot]) != cudaSuccess) {
      cudaGetLastError();
      r.state = ReqState::Failed;
      r.status = s != CABS_OK ? s : CABS_ECUDA;
      r.t_done = Clock::now();
      st->alloc.release(woff, r.ws_bytes);
      r.ws_bytes = 0;
      st->cv_done.notify_all();
      continue;
    }
    st->slot_ticket[slot] = r.ticket;
  }
}

static void serve_loop(ServeState* st) {
  cudaSetDevice(st->device);
  std::unique_lock<std::mutex> lk(st->mu);
  for (;;) {
    schedule_once(st);
    bool busy = false;
    for (uint64_t t : st->slot_ticket) busy |= t != 0;
    if (st->stopping && !busy) break;
    if (busy)
      st->cv_sched.wait_for(lk, std::chrono::microseconds(20));
    else
      st->cv_sched.wait_for(lk, std::chrono::milliseconds(5));
  }
}

}  // namespace cabs

using namespace cabs;

extern "C" {

cabs_status cabs_serve_start(cabs_ctx* ctx, void* arena, size_t arena_bytes, int32_t max_slots) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr, "ctx is NULL");
  CABS_REQUIRE(ctx->serve == nullptr, "the serving loop is already running");
  CABS_REQUIRE(arena != nullptr && ((uintptr_t)arena & 255) == 0, "arena must be non-NULL and 256-byte aligned");
  CABS_REQUIRE(arena_bytes >= 4096, "arena too small");
  CABS_REQUIRE(max_slots >= 1 && max_slots <= 64, "max_slots outside [1, 64]");
  DeviceGuard g(ctx->device);
  ServeState* st = new ServeState();
  st->arena = (char*)arena;
  st->arena_bytes = arena_bytes;
  st->device = ctx->device;
  st->alloc.reset(arena_bytes);
  for (int i = 0; i < max_slots; ++i) {
    cudaStream_t s;
    cudaEvent_t e, e0;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess) {
      for (cudaStream_t x : st->streams) cudaStreamDestroy(x);
      for (cudaEvent_t x : st->events) cudaEventDestroy(x);
      for (cudaEvent_t x : st->start_events) cudaEventDestroy(x);
      delete st;
      return check_cuda("serve stream/event");
    }
    st->streams.push_back(s);
    st->events.push_back(e);
    st->start_events.push_back(e0);
  }
  if (cudaEventCreate(&st->epoch) != cudaSuccess || cudaEventRecord(st->epoch, st->streams[0]) != cudaSuccess ||
      cudaEventSynchronize(st->epoch) != cudaSuccess) {
    for (cudaStream_t x : st->streams) cudaStreamDestroy(x);
    for (cudaEvent_t x : st->events) cudaEventDestroy(x);
    for (cudaEvent_t x : st->start_events) cudaEventDestroy(x);
    delete st;
    return check_cuda("serve epoch event");
  }
  st->slot_ticket.assign(max_slots, 0);
  st->thread = std::thread(serve_loop, st);
  ctx->serve = st;
  return CABS_OK;
}

cabs_status cabs_serve_submit(cabs_ctx* ctx, const cabs_source* src, const cabs_params* p, uint64_t* ticket) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && ctx->serve != nullptr, "the serving loop is not running");
  CABS_REQUIRE(ticket != nullptr, "ticket is NULL");
  CABS_TRY(validate_params(p));
  CABS_TRY(validate_source(src, p->m, p->n));
  CABS_REQUIRE(!(p->flags & CABS_FLAG_ERROR) || p->err_samples > 0 || src->kind != CABS_SRC_RBF,
               "the exact error needs stored entries (dense or CSR)");
  ServeState* st = ctx->serve;
  Request r;
  r.src = *src;
  r.p = *p;
  r.res_bytes = result_bytes(*p);
  r.ws_bytes = sketch_ws_bytes(*src, *p);
  r.tune = tune_lookup(ctx, *p);
  if (align256(r.res_bytes) + align256(r.ws_bytes) > st->arena_bytes) {
    set_error("request footprint %zu bytes exceeds the arena (%zu bytes)", r.res_bytes + r.ws_bytes,
              st->arena_bytes);
    return CABS_ENOMEM;
  }
  r.t_submit = Clock::now();
  {
    std::lock_guard<std::mutex> lk(st->mu);
    CABS_REQUIRE(!st->stopping, "the serving loop is stopping");
    r.ticket = st->next_ticket++;
    *ticket = r.ticket;
    st->reqs.emplace(r.ticket, r);
    st->queue.push_back(r.ticket);
  }
  st->cv_sched.notify_one();
  return CABS_OK;
}

cabs_status cabs_serve_poll(cabs_ctx* ctx, uint64_t ticket, cabs_result* res, double* latency_ms,
                            int32_t timeout_ms) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && ctx->serve != nullptr, "the serving loop is not running");
  ServeState* st = ctx->serve;
  std::unique_lock<std::mutex> lk(st->mu);
  auto it = st->reqs.find(ticket);
  if (it == st->reqs.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return CABS_ENOTFOUND;
  }
  const auto deadline = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
  while (it->second.state == ReqState::Queued || it->second.state == ReqState::Running) {
    if (timeout_ms <= 0 || st->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
      if (it->second.state == ReqState::Queued || it->second.state == ReqState::Running) return CABS_EBUSY;
    }
    it = st->reqs.find(ticket);
    if (it == st->reqs.end()) return CABS_ENOTFOUND;
  }
  const Request& r = it->second;
  if (r.state == ReqState::Failed) {
    set_error("request %llu failed with status %d", (unsigned long long)ticket, (int)r.status);
    return r.status;
  }
  if (res) *res = r.res;
  if (latency_ms) *latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  return CABS_OK;
}

cabs_status cabs_serve_times(cabs_ctx* ctx, uint64_t ticket, double* start_ms, double* end_ms) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && ctx->serve != nullptr, "the serving loop is not running");
  CABS_REQUIRE(start_ms != nullptr && end_ms != nullptr, "start_ms and end_ms must be non-NULL");
  ServeState* st = ctx->serve;
  std::lock_guard<std::mutex> lk(st->mu);
  auto it = st->reqs.find(ticket);
  if (it == st->reqs.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return CABS_ENOTFOUND;
  }
  const Request& r = it->second;
  if (r.state == ReqState::Queued || r.state == ReqState::Running) return CABS_EBUSY;
  CABS_REQUIRE(r.state == ReqState::Done && r.dev_start_ms >= 0.0, "request %llu did not finish normally",
               (unsigned long long)ticket);
  *start_ms = r.dev_start_ms;
  *end_ms = r.dev_end_ms;
  return CABS_OK;
}

cabs_status cabs_serve_release(cabs_ctx* ctx, uint64_t ticket) {
  clear_error();
  CABS_REQUIRE(ctx != nullptr && ctx->serve != nullptr, "the serving loop is not running");
  ServeState* st = ctx->serve;
  std::lock_guard<std::mutex> lk(st->mu);
  auto it = st->reqs.find(ticket);
  if (it == st->reqs.end()) {
    set_error("unknown ticket %llu", (unsigned long long)ticket);
    return CABS_ENOTFOUND;
  }
  if (it->second.state == ReqState::Queued || it->second.state == ReqState::Running) {
    set_error("request %llu has not finished", (unsigned long long)ticket);
    return CABS_EBUSY;
  }
  if (it->second.slot >= 0 || it->second.state == ReqState::Done) st->alloc.release(it->second.res_off, it->second.res_bytes);
  st->reqs.erase(it);
  return CABS_OK;
}

cabs_status cabs_serve_stop(cabs_ctx* ctx) {
  clear_error();
  if (!ctx || !ctx->serve) return CABS_OK;
  ServeState* st = ctx->serve;
  {
    std::lock_guard<std::mutex> lk(st->mu);
    st->stopping = true;
    // requests never admitted are dropped as failed
    for (uint64_t t : st->queue) {
      Request& r = st->reqs[t];
      r.state = ReqState::Failed;
      r.status = CABS_EBUSY;
    }
    st->queue.clear();
  }
  st->cv_sched.notify_all();
  if (st->thread.joinable()) st->thread.join();
  st->cv_done.notify_all();
  DeviceGuard g(st->device);
  for (cudaStream_t s : st->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : st->events) cudaEventDestroy(e);
  for (cudaEvent_t e : st->start_events) cudaEventDestroy(e);
  if (st->epoch) cudaEventDestroy(st->epoch);
  ctx->serve = nullptr;
  delete st;
  return CABS_OK;
}

}  // extern "C"
