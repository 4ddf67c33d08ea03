// Grid-wide barrier for cooperative launches, with a bounded wait (internal).
//
// All CTAs of a cooperative launch arrive on a counter; the last one bumps a
// generation word the others poll. A poll gives up after bar->limit tries
// (2^24 by default, about a second), raising bar->err so that every CTA can
// leave the kernel instead of hanging the GPU. The limit is set when the
// barrier is initialised (wait_limit(), settable through cabs_set_wait_limit
// so that tests can make a wait run out).
#pragma once

#include "common.cuh"

namespace cabs {

// Barrier state (zeroed before each launch that uses it).
struct GridBarrier {
  unsigned count;
  unsigned gen;
  int err;
  int pad;
  long long limit;  // polls before a wait gives up
};

// Poll limit for grid barriers initialised from now on (host).
long long wait_limit();

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned nblocks) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    const unsigned g = *vgen;
    __threadfence();
    ok = 1;
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      bar->count = 0u;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long spins = 0;
      const long long limit = *(volatile long long*)&bar->limit;
      while (*vgen == g) {
        if (++spins > limit || *(volatile int*)&bar->err) {
          atomicOr(&bar->err, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace cabs
