// batch_api.cu -- host runtime of genasis_batch_*: one state arena for many
// independent problems, the largest-first work list, persistent launches and
// their CUDA-graph capture, and the batch autotuner.
#include <cuda_runtime.h>

#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "aux_kernels.h"
#include "batch_kernel.cuh"
#include "batch_registry.h"
#include "common.h"
#include "genasis_hydro.h"
#include "geometry.h"

namespace gh {

__global__ void batch_finalize_kernel(int nprob, int mode, double cfl, double fixed_dt, double t_end,
                                      unsigned long long* speed, double* dt, double* t, unsigned* status) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < nprob; p += gridDim.x * blockDim.x) {
    const double s = __longlong_as_double((long long)speed[p]);
    double d = mode == FIN_CFL ? cfl / s : fixed_dt;
    const double tp = t[p];
    if (t_end > 0.0) {
      if (tp + d > t_end) d = t_end - tp;
      if (!(d > 0.0)) d = 0.0;
    }
    if (!(d >= 0.0) || !(d < INFINITY)) {
      status[p] |= STATUS_NONPHYS;
      d = 0.0;
    }
    dt[p] = d;
    t[p] = tp + d;
    speed[p] = 0ull;
  }
}

int batch_tile_count() { return 2; }

}  // namespace gh

using namespace gh;

namespace {

struct HostProblem {
  int ndim, n[2], bc_lo[2], bc_hi[2];
  double gamma;
  size_t ncell, nv, off, goff[2], woff[2];
};

}  // namespace

struct genasis_batch {
  int nprob = 0, solver = 1, prec = 0;
  double theta = 1.4;
  size_t esize = 8;
  std::vector<HostProblem> hp;
  size_t elems = 0, gelems = 0, welems = 0;
  long long cells = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  void* U[2] = {nullptr, nullptr};
  int cur = 0;
  void* K = nullptr;
  void* geo = nullptr;
  void* iw = nullptr;
  double* wd = nullptr;
  void* dprobs = nullptr;
  BatchItem* items = nullptr;
  int nitems = 0;
  unsigned* counters = nullptr;
  int ncounters = 0;
  double* dt = nullptr;
  double* t = nullptr;
  unsigned long long* speed = nullptr;
  unsigned* status = nullptr;
  int tile = 0, chunk = 32, ctas = 0;
  BatchVariant v1{}, v2{};
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int g_nsteps = -1;
  double g_cfl = 0, g_tend = 0;
};

namespace {

template <class T>
int upload_tables(genasis_batch* b, const genasis_batch_problem* probs) {
  std::vector<Geo<T>> geo;
  std::vector<T> iw;
  std::vector<double> wd;
  std::vector<BatchProblem<T>> dp(b->nprob);
  geo.reserve(b->gelems);
  iw.reserve(b->gelems);
  wd.reserve(b->welems);
  for (int p = 0; p < b->nprob; ++p) {
    const HostProblem& h = b->hp[p];
    BatchProblem<T>& d = dp[p];
    memset(&d, 0, sizeof(d));
    d.ndim = h.ndim;
    d.gamma = (T)h.gamma;
    d.gm1 = (T)(h.gamma - 1.0);
    d.off = h.off;
    for (int q = 0; q < 2; ++q) {
      d.n[q] = h.n[q];
      d.bc_lo[q] = h.bc_lo[q];
      d.bc_hi[q] = h.bc_hi[q];
      d.goff[q] = h.goff[q];
      d.woff[q] = h.woff[q];
      if (q < h.ndim) {
        append_geometry<T>(extended_widths(probs[p].widths[q], h.n[q], h.bc_lo[q], h.bc_hi[q]), b->theta, geo, iw);
        wd.insert(wd.end(), probs[p].widths[q], probs[p].widths[q] + h.n[q]);
      }
    }
  }
  GH_CK(cudaMalloc(&b->geo, geo.size() * sizeof(Geo<T>)));
  GH_CK(cudaMalloc(&b->iw, iw.size() * sizeof(T)));
  GH_CK(cudaMalloc(&b->wd, wd.size() * sizeof(double)));
  GH_CK(cudaMalloc(&b->dprobs, dp.size() * sizeof(BatchProblem<T>)));
  GH_CK(cudaMemcpy(b->geo, geo.data(), geo.size() * sizeof(Geo<T>), cudaMemcpyHostToDevice));
  GH_CK(cudaMemcpy(b->iw, iw.data(), iw.size() * sizeof(T), cudaMemcpyHostToDevice));
  GH_CK(cudaMemcpy(b->wd, wd.data(), wd.size() * sizeof(double), cudaMemcpyHostToDevice));
  GH_CK(cudaMemcpy(b->dprobs, dp.data(), dp.size() * sizeof(BatchProblem<T>), cudaMemcpyHostToDevice));
  return GENASIS_OK;
}

int configure(genasis_batch* b, int tile, int chunk) {
  if (tile < 0 || tile >= batch_tile_count()) return fail(GENASIS_EINVAL, "batch tile %d out of range", tile);
  if (chunk < 0) return fail(GENASIS_EINVAL, "chunk < 0");
  BatchVariant v1, v2;
  const bool ok =
      b->prec == GENASIS_FP64         ? batch_variant_f64(b->solver, 1, tile, &v1) && batch_variant_f64(b->solver, 2, tile, &v2)
      : b->prec == GENASIS_FP32_MIXED ? batch_variant_f32(b->solver, 1, tile, &v1) && batch_variant_f32(b->solver, 2, tile, &v2)
                                      : batch_variant_dw(b->solver, 1, tile, &v1) && batch_variant_dw(b->solver, 2, tile, &v2);
  if (!ok) return fail(GENASIS_EINVAL, "no compiled batch kernel for this configuration");
  const int cols = v1.cols;
  if (chunk == 0) chunk = 32;
  // work items: (problem, x tile, y chunk), largest first
  struct Item {
    long cost;
    BatchItem it;
  };
  std::vector<Item> items;
  for (int p = 0; p < b->nprob; ++p) {
    const HostProblem& h = b->hp[p];
    const int gx = (h.n[0] + cols - 1) / cols;
    const int gz = h.ndim == 2 ? (h.n[1] + chunk - 1) / chunk : 1;
    for (int x = 0; x < gx; ++x)
      for (int z = 0; z < gz; ++z) {
        const long w = std::min(cols, h.n[0] - x * cols);
        const long rows = h.ndim == 2 ? std::min(chunk, h.n[1] - z * chunk) + 4 : 1;
        items.push_back({w * rows, {p, x, z, 0}});
      }
  }
  std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& c) { return a.cost > c.cost; });
  std::vector<BatchItem> flat(items.size());
  for (size_t i = 0; i < items.size(); ++i) flat[i] = items[i].it;
  if (b->items) cudaFree(b->items);
  b->items = nullptr;
  GH_CK(cudaMalloc(&b->items, flat.size() * sizeof(BatchItem)));
  GH_CK(cudaMemcpy(b->items, flat.data(), flat.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  b->nitems = (int)flat.size();
  int occ1 = 0, occ2 = 0;
  for (BatchVariant* v : {&v1, &v2})
    if (v->smem > 48 * 1024) GH_CK(cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem));
  GH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, v1.fn, v1.tx, v1.smem));
  GH_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, v2.fn, v2.tx, v2.smem));
  int occ = std::max(1, std::min(occ1, occ2));
  b->ctas = std::min(b->nitems, occ * b->num_sms);
  if (b->ctas < 1) b->ctas = 1;
  b->v1 = v1;
  b->v2 = v2;
  b->tile = tile;
  b->chunk = chunk;
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
  return GENASIS_OK;
}

template <class T>
BatchArgs<T> batch_args(genasis_batch* b, int stage, unsigned* counter) {
  BatchArgs<T> A;
  A.probs = (const BatchProblem<T>*)b->dprobs;
  A.items = b->items;
  A.nitems = b->nitems;
  A.counter = counter;
  A.geo = (const Geo<T>*)b->geo;
  A.iw = (const T*)b->iw;
  A.wd = b->wd;
  A.un = (const T*)b->U[b->cur];
  A.k1 = (const T*)b->K;
  A.out = stage == 1 ? (T*)b->K : (T*)b->U[1 - b->cur];
  A.dt = b->dt;
  A.speed = b->speed;
  A.status = b->status;
  A.kchunk = b->chunk;
  return A;
}

template <class T>
int enqueue_batch_step_t(genasis_batch* b, int mode, double cfl, double t_end, unsigned* c1, unsigned* c2,
                         cudaEvent_t* ev) {
  BatchArgs<T> a1 = batch_args<T>(b, 1, c1);
  void* p1[] = {&a1};
  if (ev) GH_CK(cudaEventRecord(ev[0], b->stream));
  GH_CK(cudaLaunchKernel(b->v1.fn, dim3(b->ctas), dim3(b->v1.tx), p1, b->v1.smem, b->stream));
  if (ev) GH_CK(cudaEventRecord(ev[1], b->stream));
  const int nb = (b->nprob + 255) / 256;
  batch_finalize_kernel<<<nb, 256, 0, b->stream>>>(b->nprob, mode, cfl, 0.0, t_end, b->speed, b->dt, b->t, b->status);
  GH_CK(cudaGetLastError());
  if (ev) GH_CK(cudaEventRecord(ev[2], b->stream));
  BatchArgs<T> a2 = batch_args<T>(b, 2, c2);
  void* p2[] = {&a2};
  GH_CK(cudaLaunchKernel(b->v2.fn, dim3(b->ctas), dim3(b->v2.tx), p2, b->v2.smem, b->stream));
  if (ev) GH_CK(cudaEventRecord(ev[3], b->stream));
  b->cur = 1 - b->cur;
  return GENASIS_OK;
}

int enqueue_batch_step(genasis_batch* b, double cfl, double t_end, unsigned* c1, unsigned* c2,
                       cudaEvent_t* ev = nullptr) {
  return b->prec == GENASIS_FP64         ? enqueue_batch_step_t<double>(b, FIN_CFL, cfl, t_end, c1, c2, ev)
         : b->prec == GENASIS_FP32_MIXED ? enqueue_batch_step_t<float>(b, FIN_CFL, cfl, t_end, c1, c2, ev)
                                         : enqueue_batch_step_t<dw>(b, FIN_CFL, cfl, t_end, c1, c2, ev);
}

int ensure_counters(genasis_batch* b, int n) {
  if (n <= b->ncounters) return GENASIS_OK;
  if (b->counters) cudaFree(b->counters);
  b->counters = nullptr;
  GH_CK(cudaMalloc(&b->counters, (size_t)n * sizeof(unsigned)));
  b->ncounters = n;
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
  b->g_nsteps = -1;
  return GENASIS_OK;
}

int run_steps(genasis_batch* b, int nsteps, double cfl, double t_end) {
  int rc = ensure_counters(b, 2 * nsteps);
  if (rc) return rc;
  if (b->g_nsteps != nsteps || b->g_cfl != cfl || b->g_tend != t_end) {
    for (int k = 0; k < 2; ++k)
      if (b->graph[k]) {
        cudaGraphExecDestroy(b->graph[k]);
        b->graph[k] = nullptr;
      }
    b->g_nsteps = nsteps;
    b->g_cfl = cfl;
    b->g_tend = t_end;
  }
  const int cur0 = b->cur;
  if (!b->graph[cur0]) {
    cudaGraph_t g;
    GH_CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(b->counters, 0, (size_t)2 * nsteps * sizeof(unsigned), b->stream);
    if (e != cudaSuccess) rc = fail(GENASIS_ECUDA, "counter reset: %s", cudaGetErrorString(e));
    for (int s = 0; s < nsteps && !rc; ++s)
      rc = enqueue_batch_step(b, cfl, t_end, b->counters + 2 * s, b->counters + 2 * s + 1);
    e = cudaStreamEndCapture(b->stream, &g);
    b->cur = cur0;
    if (rc) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      return rc;
    }
    GH_CK(e);
    e = cudaGraphInstantiate(&b->graph[cur0], g, 0);
    cudaGraphDestroy(g);
    GH_CK(e);
  }
  GH_CK(cudaGraphLaunch(b->graph[cur0], b->stream));
  b->cur = cur0 ^ (nsteps & 1);
  return GENASIS_OK;
}

int free_batch(genasis_batch* b) {
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
  for (void* p : {b->U[0], b->U[1], b->K, b->geo, b->iw, (void*)b->wd, b->dprobs, (void*)b->items,
                  (void*)b->counters, (void*)b->dt, (void*)b->t, (void*)b->speed, (void*)b->status})
    if (p) cudaFree(p);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
  return GENASIS_OK;
}

}  // namespace

extern "C" {

int genasis_batch_create(int nprob, const genasis_batch_problem* probs, int solver, double theta, int precision,
                         void* stream, genasis_batch_t* out) {
  if (!out) return fail(GENASIS_EINVAL, "out is NULL");
  *out = nullptr;
  if (nprob < 1 || !probs) return fail(GENASIS_EINVAL, "need at least one problem");
  if (solver != GENASIS_HLL && solver != GENASIS_HLLC) return fail(GENASIS_EINVAL, "bad solver");
  if (!(theta >= 1.0 && theta <= 2.0)) return fail(GENASIS_EINVAL, "theta must lie in [1, 2]");
  if (precision != GENASIS_FP64 && precision != GENASIS_FP32_MIXED && precision != GENASIS_FP64_DW)
    return fail(GENASIS_EINVAL, "bad precision");
  genasis_batch* b = new genasis_batch();
  b->nprob = nprob;
  b->solver = solver;
  b->theta = theta;
  b->prec = precision;
  b->esize = precision == GENASIS_FP32_MIXED ? 4 : 8;
  b->hp.resize(nprob);
  for (int p = 0; p < nprob; ++p) {
    const genasis_batch_problem& d = probs[p];
    HostProblem& h = b->hp[p];
    memset(&h, 0, sizeof(h));
    if (d.ndim < 1 || d.ndim > 2) {
      delete b;
      return fail(GENASIS_EINVAL, "problem %d: ndim must be 1 or 2", p);
    }
    if (!(d.gamma > 1.0) || !isfinite(d.gamma)) {
      delete b;
      return fail(GENASIS_EINVAL, "problem %d: gamma must be > 1", p);
    }
    h.ndim = d.ndim;
    h.gamma = d.gamma;
    h.ncell = 1;
    for (int q = 0; q < 2; ++q) {
      const bool active = q < d.ndim;
      h.n[q] = active ? d.n[q] : 1;
      h.bc_lo[q] = active ? d.bc_lo[q] : GENASIS_BC_OUTFLOW;
      h.bc_hi[q] = active ? d.bc_hi[q] : GENASIS_BC_OUTFLOW;
      if (!active) continue;
      const char* why = nullptr;
      if (d.n[q] < 2) why = "needs at least 2 cells";
      else if (!d.widths[q]) why = "widths is NULL";
      else if (d.bc_lo[q] < 0 || d.bc_lo[q] > 2 || d.bc_hi[q] < 0 || d.bc_hi[q] > 2) why = "bad boundary code";
      else if ((d.bc_lo[q] == GENASIS_BC_PERIODIC) != (d.bc_hi[q] == GENASIS_BC_PERIODIC))
        why = "periodic must be set on both ends";
      else
        for (int i = 0; i < d.n[q] && !why; ++i)
          if (!(d.widths[q][i] > 0.0) || !isfinite(d.widths[q][i])) why = "non-positive width";
      if (why) {
        delete b;
        return fail(GENASIS_EINVAL, "problem %d axis %d: %s", p, q, why);
      }
      h.ncell *= (size_t)d.n[q];
      h.goff[q] = b->gelems;
      h.woff[q] = b->welems;
      b->gelems += d.n[q] + 4;
      b->welems += d.n[q];
    }
    h.nv = d.ndim + 2;
    h.off = b->elems;
    b->elems += h.ncell * h.nv;
    b->cells += (long long)h.ncell;
  }
#define BCK(call)                                                                                   \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      int code_ = fail(e_ == cudaErrorMemoryAllocation ? GENASIS_ENOMEM : GENASIS_ECUDA, "%s: %s", #call, \
                       cudaGetErrorString(e_));                                                     \
      free_batch(b);                                                                                \
      return code_;                                                                                 \
    }                                                                                               \
  } while (0)
  int dev = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  for (int k = 0; k < 2; ++k) {
    BCK(cudaMalloc(&b->U[k], b->elems * b->esize));
    BCK(cudaMemsetAsync(b->U[k], 0, b->elems * b->esize, b->stream));
  }
  BCK(cudaMalloc(&b->K, b->elems * b->esize));
  BCK(cudaMalloc(&b->dt, nprob * sizeof(double)));
  BCK(cudaMalloc(&b->t, nprob * sizeof(double)));
  BCK(cudaMalloc(&b->speed, nprob * sizeof(unsigned long long)));
  BCK(cudaMalloc(&b->status, nprob * sizeof(unsigned)));
  BCK(cudaMemsetAsync(b->dt, 0, nprob * sizeof(double), b->stream));
  BCK(cudaMemsetAsync(b->t, 0, nprob * sizeof(double), b->stream));
  BCK(cudaMemsetAsync(b->speed, 0, nprob * sizeof(unsigned long long), b->stream));
  BCK(cudaMemsetAsync(b->status, 0, nprob * sizeof(unsigned), b->stream));
  int rc = b->prec == GENASIS_FP64         ? upload_tables<double>(b, probs)
           : b->prec == GENASIS_FP32_MIXED ? upload_tables<float>(b, probs)
                                           : upload_tables<dw>(b, probs);
  if (!rc) rc = configure(b, 0, 0);
  if (rc) {
    free_batch(b);
    return rc;
  }
  BCK(cudaStreamSynchronize(b->stream));
#undef BCK
  *out = b;
  return GENASIS_OK;
}

int genasis_batch_destroy(genasis_batch_t b) {
  if (!b) return GENASIS_OK;
  return free_batch(b);
}

int genasis_batch_set_primitive(genasis_batch_t b, int iprob, const double* rho, const double* vel, const double* p) {
  if (!b || !rho || !vel || !p) return fail(GENASIS_EINVAL, "NULL argument");
  if (iprob < 0 || iprob >= b->nprob) return fail(GENASIS_EINVAL, "problem index out of range");
  const HostProblem& h = b->hp[iprob];
  const double* src[3] = {rho, vel, p};
  const size_t cnt[3] = {h.ncell, h.ncell * h.ndim, h.ncell};
  double* tmp[3] = {nullptr, nullptr, nullptr};
  const double* use[3];
  bool host = false;
  int rc = GENASIS_OK;
  for (int a = 0; a < 3; ++a) {
    use[a] = src[a];
    if (is_device_ptr(src[a])) continue;
    host = true;
    cudaError_t e = cudaMallocAsync((void**)&tmp[a], cnt[a] * sizeof(double), b->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(tmp[a], src[a], cnt[a] * sizeof(double), cudaMemcpyHostToDevice, b->stream);
    if (e != cudaSuccess) rc = fail(GENASIS_ECUDA, "staging primitives: %s", cudaGetErrorString(e));
    use[a] = tmp[a];
  }
  if (!rc) {
    cudaError_t e =
        b->prec == GENASIS_FP64
            ? launch_init_from_primitive<double>(h.ndim, h.ncell, h.gamma, use[0], use[1], use[2],
                                                 (double*)b->U[b->cur] + h.off, b->stream)
        : b->prec == GENASIS_FP32_MIXED
            ? launch_init_from_primitive<float>(h.ndim, h.ncell, h.gamma, use[0], use[1], use[2],
                                                (float*)b->U[b->cur] + h.off, b->stream)
            : launch_init_from_primitive<dw>(h.ndim, h.ncell, h.gamma, use[0], use[1], use[2], (dw*)b->U[b->cur] + h.off,
                                             b->stream);
    if (e != cudaSuccess) rc = fail(GENASIS_ECUDA, "init kernel: %s", cudaGetErrorString(e));
  }
  for (int a = 0; a < 3; ++a)
    if (tmp[a]) cudaFreeAsync(tmp[a], b->stream);
  if (rc) return rc;
  GH_CK(cudaMemsetAsync(b->t + iprob, 0, sizeof(double), b->stream));
  if (host) GH_CK(cudaStreamSynchronize(b->stream));
  return GENASIS_OK;
}

int genasis_batch_get_conserved(genasis_batch_t b, int iprob, void* U, int precision) {
  if (!b || !U) return fail(GENASIS_EINVAL, "NULL argument");
  if (iprob < 0 || iprob >= b->nprob) return fail(GENASIS_EINVAL, "problem index out of range");
  if (precision != GENASIS_FP64 && precision != GENASIS_FP32_MIXED) return fail(GENASIS_EINVAL, "bad precision");
  const HostProblem& h = b->hp[iprob];
  const size_t count = h.ncell * h.nv;
  const bool dev = is_device_ptr(U);
  const char* src = (const char*)b->U[b->cur] + h.off * b->esize;
  if (precision == b->prec) {
    GH_CK(cudaMemcpyAsync(U, src, count * b->esize, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  } else {
    const size_t dsize = precision == GENASIS_FP64 ? 8 : 4;
    void* dst = U;
    if (!dev) GH_CK(cudaMallocAsync(&dst, count * dsize, b->stream));
    cudaError_t e;
    if (b->prec == GENASIS_FP64_DW)
      e = precision == GENASIS_FP64 ? launch_convert<dw, double>(count, (const dw*)src, (double*)dst, b->stream)
                                    : launch_convert<dw, float>(count, (const dw*)src, (float*)dst, b->stream);
    else
      e = b->prec == GENASIS_FP64 ? launch_convert<double, float>(count, (const double*)src, (float*)dst, b->stream)
                                  : launch_convert<float, double>(count, (const float*)src, (double*)dst, b->stream);
    GH_CK(e);
    if (!dev) {
      GH_CK(cudaMemcpyAsync(U, dst, count * dsize, cudaMemcpyDeviceToHost, b->stream));
      GH_CK(cudaFreeAsync(dst, b->stream));
    }
  }
  GH_CK(cudaStreamSynchronize(b->stream));
  return GENASIS_OK;
}

int genasis_batch_run(genasis_batch_t b, int nsteps, double cfl, double t_end) {
  if (!b) return fail(GENASIS_EINVAL, "NULL batch");
  if (nsteps < 0) return fail(GENASIS_EINVAL, "nsteps < 0");
  if (!(cfl > 0.0)) return fail(GENASIS_EINVAL, "cfl must be > 0");
  if (nsteps == 0) return GENASIS_OK;
  return run_steps(b, nsteps, cfl, t_end);
}

int genasis_batch_get_times(genasis_batch_t b, double* t) {
  if (!b || !t) return fail(GENASIS_EINVAL, "NULL argument");
  GH_CK(cudaMemcpyAsync(t, b->t, b->nprob * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  GH_CK(cudaStreamSynchronize(b->stream));
  return GENASIS_OK;
}

int genasis_batch_status(genasis_batch_t b, int* first_bad) {
  if (!b) return fail(GENASIS_EINVAL, "NULL batch");
  std::vector<unsigned> st(b->nprob);
  GH_CK(cudaMemcpyAsync(st.data(), b->status, b->nprob * sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
  GH_CK(cudaStreamSynchronize(b->stream));
  int bad = -1;
  for (int p = 0; p < b->nprob && bad < 0; ++p)
    if (st[p]) bad = p;
  if (first_bad) *first_bad = bad;
  if (bad >= 0) return fail(GENASIS_ENONPHYS, "problem %d met a non-physical state", bad);
  return GENASIS_OK;
}

int genasis_batch_set_tile(genasis_batch_t b, int tile, int chunk) {
  if (!b) return fail(GENASIS_EINVAL, "NULL batch");
  GH_CK(cudaStreamSynchronize(b->stream));
  return configure(b, tile, chunk);
}

int genasis_batch_get_tile(genasis_batch_t b, int* info) {
  if (!b || !info) return fail(GENASIS_EINVAL, "NULL argument");
  info[0] = b->tile;
  info[1] = b->v1.tx;
  info[2] = b->chunk;
  info[3] = b->nitems;
  info[4] = b->ctas;
  info[5] = batch_tile_count();
  info[6] = (int)(b->cells >> 20);
  return GENASIS_OK;
}

int genasis_batch_profile_step(genasis_batch_t b, double cfl, float* ms) {
  if (!b || !ms) return fail(GENASIS_EINVAL, "NULL argument");
  int rc = ensure_counters(b, 2);
  if (rc) return rc;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int i = 0; i < 4 && !rc; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = fail(GENASIS_ECUDA, "cudaEventCreate failed");
  if (!rc && cudaMemsetAsync(b->counters, 0, 2 * sizeof(unsigned), b->stream) != cudaSuccess)
    rc = fail(GENASIS_ECUDA, "counter reset failed");
  if (!rc) rc = enqueue_batch_step(b, cfl, 0.0, b->counters, b->counters + 1, ev);
  if (!rc && cudaEventSynchronize(ev[3]) != cudaSuccess) rc = fail(GENASIS_ECUDA, "profile sync failed");
  if (!rc) {
    cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
    cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
    cudaEventElapsedTime(&ms[2], ev[2], ev[3]);
  }
  for (int i = 0; i < 4; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  return rc;
}

int genasis_batch_autotune(genasis_batch_t b, int trial_steps, const char* cache_path) {
  if (!b || trial_steps < 1) return fail(GENASIS_EINVAL, "bad argument");
  char key[160];
  snprintf(key, sizeof(key), "batch nprob=%d cells=%lld prec=%d solver=%d", b->nprob, b->cells, b->prec, b->solver);
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[256];
      int tile = -1, ch = -1;
      const size_t kl = strlen(key);
      while (fgets(line, sizeof(line), f)) {
        int t2, c2;
        if (strncmp(line, key, kl) == 0 && line[kl] == ' ' && sscanf(line + kl, " tile=%d chunk=%d", &t2, &c2) == 2) {
          tile = t2;
          ch = c2;
        }
      }
      fclose(f);
      if (tile >= 0 && tile < batch_tile_count()) return configure(b, tile, ch);
    }
  }
  const size_t bytes = b->elems * b->esize;
  void* save = nullptr;
  GH_CK(cudaMalloc(&save, bytes));
  std::vector<double> tsave(b->nprob);
  GH_CK(cudaMemcpyAsync(save, b->U[b->cur], bytes, cudaMemcpyDeviceToDevice, b->stream));
  GH_CK(cudaMemcpyAsync(tsave.data(), b->t, b->nprob * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  GH_CK(cudaStreamSynchronize(b->stream));
  const int cur_save = b->cur;
  cudaEvent_t e0, e1;
  GH_CK(cudaEventCreate(&e0));
  GH_CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_tile = 0, best_chunk = 32, rc = GENASIS_OK;
  for (int tile = 0; tile < batch_tile_count() && !rc; ++tile)
    for (int ch : {16, 32, 64, 128, 256}) {
      rc = configure(b, tile, ch);
      if (!rc) rc = run_steps(b, 1, 0.1, 0.0);  // warm-up and capture
      if (!rc) {
        cudaEventRecord(e0, b->stream);
        for (int s = 0; s < trial_steps && !rc; ++s) rc = run_steps(b, 1, 0.1, 0.0);
        cudaEventRecord(e1, b->stream);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(GENASIS_ECUDA, "autotune timing failed");
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (!rc && ms < best) {
          best = ms;
          best_tile = tile;
          best_chunk = ch;
        }
      }
      b->cur = cur_save;
      cudaMemcpyAsync(b->U[b->cur], save, bytes, cudaMemcpyDeviceToDevice, b->stream);
      if (rc) break;
    }
  cudaMemcpyAsync(b->t, tsave.data(), b->nprob * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  cudaMemsetAsync(b->status, 0, b->nprob * sizeof(unsigned), b->stream);
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = configure(b, best_tile, best_chunk);
  if (rc) return rc;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "%s tile=%d chunk=%d ms_per_step=%.6f\n", key, best_tile, best_chunk, best / trial_steps);
      fclose(f);
    }
  }
  return GENASIS_OK;
}

}  // extern "C"
