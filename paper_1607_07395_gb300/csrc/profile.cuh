// Kernel timing scopes and the launch counter (internal).
#pragma once

#include "common.cuh"

namespace cabs {

// Records CUDA events around the enclosed launch when profiling is on.
class ProfScope {
 public:
  ProfScope(cudaStream_t s, const char* name);
  ~ProfScope();
  ProfScope(const ProfScope&) = delete;
  ProfScope& operator=(const ProfScope&) = delete;

 private:
  cudaStream_t stream_;
  const char* name_;
  cudaEvent_t a_;
};

// Counts one kernel launch and converts a launch error into CABS_ECUDA.
cabs_status launched(const char* what);

// Launches counted on the calling thread so far (graph capture bookkeeping).
long long thread_launches();
// Adds n to the launch counter (n < 0 removes launches that were only captured).
void add_launches(long long n);

}  // namespace cabs

// Wraps one kernel launch statement: times it (when enabled), counts it,
// checks it, and returns from the enclosing function on failure.
#define CABS_LAUNCH(stream, name, ...)           \
  do {                                           \
    {                                            \
      ::cabs::ProfScope _ps((stream), (name));   \
      __VA_ARGS__;                               \
    }                                            \
    CABS_TRY(::cabs::launched(name));            \
  } while (0)
