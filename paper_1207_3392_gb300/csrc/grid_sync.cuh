// grid_sync.cuh -- a bounded barrier over all CTAs of a cooperative launch,
// used by the kernels that run several dependent phases (or whole steps) in
// one launch.
//
// The barrier is a counter and a generation word in device memory, both zero
// before the launch.  The last CTA to arrive resets the counter and moves the
// generation on; the others poll the generation word with __nanosleep between
// polls.  A wait is bounded by about one second of %globaltimer: a CTA that
// gives up sets STATUS_TIMEOUT in *status and leaves, and every CTA leaves at
// its next barrier, so the launch ends instead of hanging.
#pragma once

#include "hydro_device.cuh"

namespace gh {

__device__ __forceinline__ unsigned long long global_timer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Barrier of all nblocks CTAs of the launch; false (on every thread of the
// CTA) if this CTA gave up waiting here or at an earlier barrier.  my_gen is
// the generation this CTA last saw (read from gen at launch by thread 0).
__device__ inline bool grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, unsigned& my_gen, unsigned* status,
                                    bool& failed) {
  __syncthreads();
  if (threadIdx.x == 0 && !failed) {
    __threadfence();  // this CTA's writes before the arrival
    const unsigned g = my_gen;
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicExch(gen, g + 1u);
    } else {
      const unsigned long long t0 = global_timer_ns();
      while (atomicAdd(gen, 0u) == g) {
        if (global_timer_ns() - t0 > 1000000000ull) {
          failed = true;
          atomicOr(status, STATUS_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();  // the others' writes after the release
    my_gen = g + 1u;
  }
  return __syncthreads_or(failed ? 1 : 0) == 0;
}

}  // namespace gh
