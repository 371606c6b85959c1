// peak_probe.cu -- genasis_measure_fma_rate: the vector FMA throughput of the
// current GPU, measured with independent FMA chains (the denominator of the
// arithmetic roofline of the stage kernels); genasis_measure_link_rate: the
// host-link copy rate (the denominator of the end-to-end roofline).  Not
// part of the update.
#include <cuda_runtime.h>

#include <string.h>

#include "common.h"
#include "genasis_hydro.h"

namespace {

constexpr int CHAINS = 8;     // independent accumulators per thread
constexpr int THREADS = 256;

// acc <- acc * b + c on CHAINS independent accumulators; b < 1 and c small
// keep the values bounded.  Every accumulator is summed into out so that no
// chain is dead code.
template <class T>
__global__ void __launch_bounds__(THREADS) fma_chain_kernel(T b, T c, int iters, T* out) {
  T acc[CHAINS];
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) acc[j] = (T)(threadIdx.x + j) * (T)1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) acc[j] = fma(acc[j], b, c);
  }
  T s = (T)0;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) s += acc[j];
  out[(size_t)blockIdx.x * THREADS + threadIdx.x] = s;
}

// The same with the packed FP32 pair instruction of sm_100+ (two FMAs per
// instruction on a 64-bit register pair).
__global__ void __launch_bounds__(THREADS) fma_chain_f32x2_kernel(float b, float c, int iters, float* out) {
  unsigned long long acc[CHAINS];
  const float2 bb = make_float2(b, b), cc = make_float2(c, c);
  unsigned long long bp, cp;
  memcpy(&bp, &bb, 8);
  memcpy(&cp, &cc, 8);
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) {
    const float2 v = make_float2((float)(threadIdx.x + j) * 1e-3f, (float)(threadIdx.x + 2 * j) * 1e-3f);
    memcpy(&acc[j], &v, 8);
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < CHAINS; ++j) asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(acc[j]) : "l"(bp), "l"(cp));
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < CHAINS; ++j) {
    float2 v;
    memcpy(&v, &acc[j], 8);
    s += v.x + v.y;
  }
  out[(size_t)blockIdx.x * THREADS + threadIdx.x] = s;
}

}  // namespace

extern "C" int genasis_measure_fma_rate(int kind, double* tflops) {
  if (!tflops || kind < 0 || kind > 2) return gh::fail(GENASIS_EINVAL, "measure_fma_rate: bad argument");
  int dev = 0, sms = 0;
  GH_CK(cudaGetDevice(&dev));
  GH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = sms * 8;  // 8 CTAs of 256 threads per SM: every SM full
  const int iters = kind == 0 ? 1 << 6 : 1 << 11;  // ~0.1-0.3 s per launch
  void* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = GENASIS_OK;
  float ms = 0.0f;
  cudaError_t e = cudaMalloc(&out, (size_t)blocks * THREADS * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first launch warms up
    e = cudaEventRecord(e0, st);
    if (kind == 0) fma_chain_kernel<double><<<blocks, THREADS, 0, st>>>(0.999999, 1e-7, iters, (double*)out);
    else if (kind == 1) fma_chain_kernel<float><<<blocks, THREADS, 0, st>>>(0.9999f, 1e-5f, iters, (float*)out);
    else fma_chain_f32x2_kernel<<<blocks, THREADS, 0, st>>>(0.9999f, 1e-5f, iters, (float*)out);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  }
  if (e != cudaSuccess) rc = gh::fail(GENASIS_ECUDA, "measure_fma_rate: %s", cudaGetErrorString(e));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  if (rc) return rc;
  const double fmas = (double)blocks * THREADS * CHAINS * iters * (kind == 2 ? 2.0 : 1.0);
  *tflops = 2.0 * fmas / (ms * 1e-3) / 1e12;
  return GENASIS_OK;
}

// Host-link copy rate (the denominator of the end-to-end roofline): 256 MiB
// page-locked host buffers and device buffers, copied with cudaMemcpyAsync on
// private streams, kind 0 host to device, 1 device to host, 2 both directions
// at once on two streams (GB/s of the two together).  One warm-up, then the
// mean of four timed copies.
extern "C" int genasis_measure_link_rate(int kind, double* gbs) {
  if (!gbs || kind < 0 || kind > 2) return gh::fail(GENASIS_EINVAL, "measure_link_rate: bad argument");
  const size_t bytes = (size_t)256 << 20;
  void *h_in = nullptr, *h_out = nullptr, *d_a = nullptr, *d_b = nullptr;
  cudaStream_t s[2] = {nullptr, nullptr};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.0f;
  cudaError_t e = cudaHostAlloc(&h_in, bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaHostAlloc(&h_out, bytes, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaMalloc(&d_a, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&d_b, bytes);
  if (e == cudaSuccess) memset(h_in, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(d_b, 0, bytes);
  for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaStreamCreateWithFlags(&s[i], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int reps = 4;
  for (int round = 0; round < 2 && e == cudaSuccess; ++round) {  // the first round warms up
    const int n = round == 0 ? 1 : reps;
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s[0]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s[1], e0, 0);
    for (int r = 0; r < n && e == cudaSuccess; ++r) {
      if (kind != 1) e = cudaMemcpyAsync(d_a, h_in, bytes, cudaMemcpyHostToDevice, s[0]);
      if (kind != 0 && e == cudaSuccess) e = cudaMemcpyAsync(h_out, d_b, bytes, cudaMemcpyDeviceToHost, s[1]);
    }
    // the end event on s[0] after s[1]'s copies too
    cudaEvent_t join = nullptr;
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(join, s[1]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s[0], join, 0);
    if (e == cudaSuccess) e = cudaEventRecord(e1, s[0]);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (join) cudaEventDestroy(join);
  }
  const int rc = e == cudaSuccess ? GENASIS_OK : gh::fail(GENASIS_ECUDA, "measure_link_rate: %s", cudaGetErrorString(e));
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int i = 0; i < 2; ++i)
    if (s[i]) cudaStreamDestroy(s[i]);
  cudaFreeHost(h_in);
  cudaFreeHost(h_out);
  cudaFree(d_a);
  cudaFree(d_b);
  if (rc) return rc;
  *gbs = (kind == 2 ? 2.0 : 1.0) * (double)bytes * reps / (ms * 1e-3) / 1e9;
  return GENASIS_OK;
}
