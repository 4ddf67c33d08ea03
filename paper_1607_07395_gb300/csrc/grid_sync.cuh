// Grid-wide barrier for cooperative launches, with a bounded wait (internal).
//
// All CTAs of a cooperative launch arrive on a counter; the last one bumps a
// generation word the others poll. A poll gives up after ~2^24 tries (about a
// second), raising bar->err so that every CTA can leave the kernel instead of
// hanging the GPU.
#pragma once

#include "common.cuh"

namespace cabs {

// Barrier state (zeroed before each launch that uses it).
struct GridBarrier {
  unsigned count;
  unsigned gen;
  int err;
};

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
      while (*vgen == g) {
        if (++spins > (1ll << 24) || *(volatile int*)&bar->err) {
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
