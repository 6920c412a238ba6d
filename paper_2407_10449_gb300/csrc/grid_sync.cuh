// grid_sync.cuh -- a bounded grid-wide barrier for persistent cooperative
// kernels (every CTA of the launch co-resident).  Internal to each
// translation unit that includes it.
#pragma once

#include <cstdint>

#include "ess_common.cuh"

namespace ess {
namespace {

__device__ __forceinline__ unsigned long long grid_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier over all CTAs of the cooperative launch (all co-resident):
// arrivals counted in bar[0], release by bumping the generation in bar[1].  A
// wait longer than wait_ns sets the time-out status and the abort flag.
// withhold: this CTA waits without arriving (the self-test of the bound).
// Returns false if the run is aborted (every CTA then leaves at this point).
__device__ bool grid_barrier(unsigned* bar, int* abort_flag, int* status,
                             unsigned long long wait_ns, bool withhold = false) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* gen = bar + 1;
    const unsigned g = *gen;
    __threadfence();
    bool ok = true;
    if (!withhold && atomicAdd(bar, 1u) == gridDim.x - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const unsigned long long t0 = grid_now();
      int spins = 0;
      while (*gen == g) {
        if (++spins == 64) {
          spins = 0;
          if (grid_now() - t0 > wait_ns ||
              *reinterpret_cast<volatile int*>(abort_flag) != 0) {
            ok = false;
            break;
          }
        }
      }
    }
    __threadfence();
    if (!ok) {
      atomicOr(status, kStatusTimeout);
      atomicExch(abort_flag, 1);
    }
    s_ok = ok && *reinterpret_cast<volatile int*>(abort_flag) == 0;
  }
  __syncthreads();
  return s_ok != 0;
}

}  // namespace
}  // namespace ess
