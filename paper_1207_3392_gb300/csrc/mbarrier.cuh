// mbarrier.cuh -- shared-memory barrier, proxy-fence and TMA-load helpers of
// the kernels that use the asynchronous units (TMA copies, tensor-core MMAs).
// Every wait is bounded: mbar_wait gives up after about one second.
#pragma once

#include <cuda.h>
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

// Non-blocking test of the phase (no suspend): for waits that are usually
// short, where a suspended thread would wake later than the phase completes.
__device__ __forceinline__ bool mbar_test(unsigned long long* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Spin on mbar_test; false after ~1 s.
__device__ __forceinline__ bool mbar_wait_spin(unsigned long long* b, unsigned parity) {
  if (mbar_test(b, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (!mbar_test(b, parity)) {
    if (globaltimer() - t0 > 1000000000ull) return false;
  }
  return true;
}

// Order this thread's generic-proxy accesses to shared memory before later
// async-proxy accesses to the same memory (TMA writes, tensor-core operand
// reads).
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Tiled 4D TMA load of the map's box at (x, y, z, v) into dst, counted on
// the transaction bytes of mbarrier bar.  x * element size must be a
// multiple of 16 bytes; other coordinates may lie outside the tensor (the
// box then reads the fill value there).
__device__ __forceinline__ void load_4d(void* dst, const CUtensorMap* map, int x, int y, int z, int v,
                                        unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(v), "r"(smem_u32(bar))
      : "memory");
}
// Barrier of the compute threads only (named barrier 1; the producer warp
// takes no part) that also ORs a flag over them: every thread leaves with
// the same answer, so a decision taken on it is uniform.
template <int N>
__device__ __forceinline__ bool sync_compute_or(bool flag) {
  unsigned out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(out)
      : "r"((unsigned)flag), "n"(N)
      : "memory");
  return out != 0u;
}

}  // namespace tma
}  // namespace gh
