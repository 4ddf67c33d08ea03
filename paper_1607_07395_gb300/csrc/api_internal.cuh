// Internal declarations shared by the ABI layer (api.cu) and the serving loop
// (serve.cu). Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace cabs {

// Selects a device for the lifetime of the guard and restores the previous one.
struct DeviceGuard {
  int prev = 0;
  int target = 0;
  bool ok = false;
  explicit DeviceGuard(int dev);
  ~DeviceGuard();
};

// Slices of one sketch's workspace (see carve_sketch).
struct SketchWs {
  int *pr_drawn, *pc_drawn, *fr_order, *fc_order;
  void *C, *Rt, *P, *Q, *Zr, *Zc;
  double *W, *S_pilot;
  cabs_diag* diag;
  void *core, *side_r, *side_c;
  size_t core_bytes, side_r_bytes, side_c_bytes;
  void *lev_X, *lev_Y;      // CABS_FLAG_LEVERAGE: orthonormal pilot factors
  double *lev_one, *lev_s;  //   ones (the S of P Q^T) and its singular values
  double* err_out2;  // CABS_FLAG_ERROR: (num, den) of the error
  void* err_ws;
  size_t err_bytes;
};

struct GraphEntry {
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;  // kernel launches held by the graph
};

struct ServeState;

SketchWs carve_sketch(Carve& cv, const cabs_source& src, const cabs_params& p);
size_t sketch_ws_bytes(const cabs_source& src, const cabs_params& p);
cabs_status validate_error_request(const cabs_source* src, const cabs_params* p, const cabs_result* out);
cabs_status validate_source(const cabs_source* src, int64_t m, int64_t n);
cabs_status validate_params(const cabs_params* p);
cabs_status validate_result(const cabs_result* out);
// fork_sides: run the column side of step 3 on a second stream (a sketch on
// its own; a batch's lanes already run sketches side by side)
cabs_status sketch_enqueue(const cabs_source& src, const cabs_params& p, void* ws, size_t ws_bytes, cudaStream_t s,
                           const cabs_result& out, bool fork_sides = true);
// Batched form: members largest first over `lanes` internal streams forked
// from and joined back to s (each member under its bucket's launch shape).
cabs_status ensure_lanes(cabs_ctx* ctx, int lanes);
cabs_status batched_enqueue(cabs_ctx* ctx, int count, const cabs_source* src, const cabs_params* p, void* ws,
                            const size_t* off, const cabs_result* out, int lanes, cudaStream_t s);
// The tuning-table bucket of a sketch shape and the entry in force for it.
uint32_t tune_bucket(int prec, int k, int64_t m, int64_t n);
cabs_tune tune_lookup(cabs_ctx* ctx, const cabs_params& p);

}  // namespace cabs

// The opaque context of the ABI.
struct cabs_ctx {
  int device = 0;
  // launch shapes per shape bucket (cabs_tune_set / cabs_autotune) and the
  // lanes cabs_autotune chose for batches; version bumps invalidate graphs
  std::mutex tune_mu;
  std::unordered_map<uint32_t, cabs_tune> tune;
  int tuned_lanes = 0;
  uint64_t tune_version = 0;
  std::mutex graph_mu;
  std::unordered_map<uint64_t, cabs::GraphEntry> graphs;
  std::vector<cudaStream_t> lanes;
  std::vector<cudaEvent_t> lane_events;
  cudaEvent_t fork_event = nullptr;
  cabs::ServeState* serve = nullptr;
};
