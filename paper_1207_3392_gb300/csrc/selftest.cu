// selftest.cu -- a check that the bounded waits of the kernels give up and
// report instead of hanging.  Two waits that cannot complete, each on its own
// status word:
//   grid barrier (grid_sync.cuh): of two CTAs only the first arrives, so the
//     generation word it polls never moves;
//   mbarrier (mbarrier.cuh): one thread waits on an mbarrier that nothing
//     arrives on (the kind of wait of the TMA and tcgen05 kernels).
// Each gives up after about one second and sets STATUS_TIMEOUT; the launches
// end normally and the context stays usable.  Nothing faults or traps.
#include <cuda_runtime.h>

#include "common.h"
#include "genasis_hydro.h"
#include "grid_sync.cuh"
#include "mbarrier.cuh"

namespace gh {
namespace {

__global__ void barrier_wait_probe(unsigned* words, unsigned* status) {
  if (blockIdx.x != 0) return;  // the second CTA never arrives
  unsigned my_gen = 0;
  bool failed = false;
  grid_barrier(words, words + 1, 2u, my_gen, status, failed);
}

__global__ void mbarrier_wait_probe(unsigned* status) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) {
    tma::mbar_init(&bar, 1);
    tma::fence_mbar_init();
    if (!tma::mbar_wait(&bar, 0)) atomicOr(status, STATUS_TIMEOUT);  // nothing arrives
  }
}

}  // namespace
}  // namespace gh

using namespace gh;

extern "C" int genasis_check_bounded_waits(unsigned* status, double* seconds) {
  if (!status || !seconds) return fail(GENASIS_EINVAL, "check_bounded_waits: NULL argument");
  unsigned* d = nullptr;
  cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
  int rc = GENASIS_OK;
  cudaError_t err = cudaMalloc((void**)&d, 4 * sizeof(unsigned));
  for (int i = 0; i < 3 && err == cudaSuccess; ++i) err = cudaEventCreate(&e[i]);
  if (err == cudaSuccess) err = cudaMemset(d, 0, 4 * sizeof(unsigned));
  if (err == cudaSuccess) {
    // d[0..1]: barrier count and generation; d[2], d[3]: the two status words
    cudaEventRecord(e[0]);
    barrier_wait_probe<<<2, 32>>>(d, d + 2);
    cudaEventRecord(e[1]);
    mbarrier_wait_probe<<<1, 32>>>(d + 3);
    cudaEventRecord(e[2]);
    err = cudaGetLastError();
  }
  unsigned host[4] = {0, 0, 0, 0};
  if (err == cudaSuccess) err = cudaMemcpy(host, d, sizeof(host), cudaMemcpyDeviceToHost);
  if (err == cudaSuccess) {
    float ms0 = 0.0f, ms1 = 0.0f;
    cudaEventElapsedTime(&ms0, e[0], e[1]);
    cudaEventElapsedTime(&ms1, e[1], e[2]);
    status[0] = host[2];
    status[1] = host[3];
    seconds[0] = ms0 * 1e-3;
    seconds[1] = ms1 * 1e-3;
  } else {
    rc = fail(GENASIS_ECUDA, "check_bounded_waits: %s", cudaGetErrorString(err));
  }
  for (int i = 0; i < 3; ++i)
    if (e[i]) cudaEventDestroy(e[i]);
  cudaFree(d);
  return rc;
}
