// mbarrier.cuh -- shared-memory barrier and proxy-fence helpers of the
// kernels that use the asynchronous units (TMA copies, tensor-core MMAs).
// Every wait is bounded: mbar_wait gives up after about one second.
#pragma once

#include <cuda_runtime.h>

namespace gh {
namespace tma {

__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// One test of the phase, with a suspend-time hint: the thread may sleep in
// hardware (issuing nothing) until the phase completes or ~0.1 ms pass.
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for the phase of parity `parity` to complete; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
  if (mbar_try(b, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_try(b, parity)) {
    if (globaltimer() - t0 > 1000000000ull) return false;
  }
  return true;
}

// Order this thread's generic-proxy accesses to shared memory before later
// async-proxy accesses to the same memory (TMA writes, tensor-core operand
// reads).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

}  // namespace tma
}  // namespace gh
