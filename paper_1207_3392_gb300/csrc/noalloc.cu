// noalloc.cu -- genasis_hydro_step_noalloc: one RK2 step that allocates no
// memory.  For callers that cannot call cudaMalloc -- code whose device memory
// is owned by a pooling allocator that has already reserved it (a cudaMalloc
// there fails or fragments the pool), and latency-critical loops that must not
// allocate after initialisation (cudaMalloc may synchronise the device).
//
// The stage buffer, the reduction partials, the device scalars and the
// geometry tables live in one file-scope device array, g_noalloc_scratch, of
// NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds that array
// until the process exits.  Every call shares it: concurrent calls (on
// different streams, or from different host threads) race on it, and it keeps
// the contents of the last call.
#include <cuda_runtime.h>

#include <math.h>
#include <mutex>

#include "aux_kernels.h"
#include "common.h"
#include "genasis_hydro.h"
#include "registry.h"
#include "stage_kernel.cuh"

namespace gh {

static constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)32 << 20;  // 32 MiB
static constexpr int NOALLOC_MAX_N = 4096;                         // cells per axis
static constexpr int NOALLOC_MAX_CTAS = 4096;                      // CTAs per stage

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

// Scratch layout (byte offsets, each region 256-byte aligned).
static constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }
static constexpr size_t OFF_SCAL = 0;                                                   // SCAL_ALLOC doubles
static constexpr size_t OFF_STATUS = align256(OFF_SCAL + SCAL_ALLOC * sizeof(double));  // unsigned
static constexpr size_t OFF_SPEED = align256(OFF_STATUS + sizeof(unsigned));
static constexpr size_t OFF_TOT = align256(OFF_SPEED + NOALLOC_MAX_CTAS * sizeof(double));
static constexpr size_t GEO_N = NOALLOC_MAX_N + 4;
static constexpr size_t OFF_WD = align256(OFF_TOT + (size_t)NOALLOC_MAX_CTAS * 5 * sizeof(double));
static constexpr size_t OFF_GEO = align256(OFF_WD + 3 * NOALLOC_MAX_N * sizeof(double));
static constexpr size_t OFF_IW = align256(OFF_GEO + 3 * GEO_N * sizeof(Geo<double>));
static constexpr size_t OFF_K = align256(OFF_IW + 3 * GEO_N * sizeof(double));
static constexpr size_t K_BYTES = NOALLOC_SCRATCH_BYTES - OFF_K;

// Device address of g_noalloc_scratch per device, set up once per device.
static std::mutex g_noalloc_mutex;
static unsigned char* g_noalloc_ptr[64] = {nullptr};

// Reconstruction tables of one axis from its widths (same formulas as the
// handle set-up: two ghost widths per side by the boundary rule, centre
// distances of Eq. MinMod on a non-uniform Cartesian mesh).
template <class T>
__global__ void noalloc_geometry_kernel(int n, int lo, int hi, double theta, const double* __restrict__ w, Geo<T>* geo,
                                        T* iw) {
  const int m = n + 4;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    double e3[3];
    for (int d = -1; d <= 1; ++d) {
      int kk = k + d;
      kk = kk < 0 ? 0 : (kk > m - 1 ? m - 1 : kk);
      const int c = kk - 2;
      int s = c;
      if (c < 0) s = lo == BC_PERIODIC ? c + n : lo == BC_REFLECT ? -1 - c : 0;
      else if (c >= n) s = hi == BC_PERIODIC ? c - n : hi == BC_REFLECT ? 2 * n - 1 - c : n - 1;
      e3[d + 1] = w[s];
    }
    const double dm = e3[0], dc = e3[1], dp = e3[2];
    Geo<T> g;
    g.ticm = (T)(theta / (0.5 * (dm + dc)));
    g.ipm = (T)(1.0 / (0.5 * dm + dc + 0.5 * dp));
    g.tipc = (T)(theta / (0.5 * (dc + dp)));
    g.h = (T)(0.5 * dc);
    geo[k] = g;
    iw[k] = (T)(1.0 / dc);
  }
}

// First call on a device: look up the device address of the scratch array
// with that device current.  The address is cached for the life of the
// process; a cudaDeviceReset of that device unloads the module and leaves the
// cached address stale, so the entry point must not be used on a device after
// a reset in the same process.
static int scratch_for_current_device(unsigned char** out) {
  int dev = 0;
  GH_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(GENASIS_EINVAL, "device index %d unsupported", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    GH_CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = (unsigned char*)p;
  }
  *out = g_noalloc_ptr[dev];
  return GENASIS_OK;
}

template <class T>
static int noalloc_step_t(const genasis_hydro_desc* d, unsigned char* base, const T* uin, T* uout, double dt,
                          cudaStream_t st) {
  const int ndim = d->ndim;
  int n[3] = {1, 1, 1}, lo[3] = {BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW}, hi[3] = {BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW};
  size_t ncell = 1;
  for (int q = 0; q < ndim; ++q) {
    n[q] = d->n[q];
    lo[q] = d->bc_lo[q];
    hi[q] = d->bc_hi[q];
    ncell *= (size_t)n[q];
  }
  const size_t nv = (size_t)ndim + 2;
  if (ncell * nv * sizeof(T) > K_BYTES)
    return fail(GENASIS_EINVAL, "step_noalloc: %zu cells x %zu variables x %zu bytes exceeds the %zu-byte scratch stage buffer",
                ncell, nv, sizeof(T), K_BYTES);
  // launch configuration: tile 0, about four CTAs per SM, at least 8 planes per CTA
  StageVariant v1, v2;
  const bool fp64 = sizeof(T) == 8;
  const int prec = fp64 ? GENASIS_FP64 : GENASIS_FP32_MIXED;
  if (!stage_variant(ndim, prec, d->solver, 1, 0, &v1) || !stage_variant(ndim, prec, d->solver, 2, 0, &v2))
    return fail(GENASIS_EINVAL, "step_noalloc: no compiled kernel for this configuration");
  int dev = 0, sms = 0;
  GH_CK(cudaGetDevice(&dev));
  GH_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int gx = (n[0] + v1.tx - 1) / v1.tx;
  const int gy = ndim == 3 ? (n[1] + v1.ty - 1) / v1.ty : 1;
  const int nm = ndim >= 2 ? n[ndim - 1] : 1;
  int kchunk = 1, gz = 1;
  if (ndim >= 2) {
    long chunks = (4L * sms + (long)gx * gy - 1) / ((long)gx * gy);
    const long maxchunks = nm / 8 > 0 ? nm / 8 : 1;
    chunks = chunks > maxchunks ? maxchunks : (chunks < 1 ? 1 : chunks);
    while ((long)gx * gy * chunks > NOALLOC_MAX_CTAS && chunks > 1) --chunks;
    kchunk = (int)((nm + chunks - 1) / chunks);
    gz = (nm + kchunk - 1) / kchunk;
  }
  const long nblk = (long)gx * gy * gz;
  if (nblk > NOALLOC_MAX_CTAS)
    return fail(GENASIS_EINVAL, "step_noalloc: %ld CTAs per stage exceed the limit of %d", nblk, NOALLOC_MAX_CTAS);
  for (const StageVariant* v : {&v1, &v2})
    if (v->smem > 48 * 1024) GH_CK(cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem));

  double* scal = (double*)(base + OFF_SCAL);
  unsigned* status = (unsigned*)(base + OFF_STATUS);
  double* speed = (double*)(base + OFF_SPEED);
  double* tot = (double*)(base + OFF_TOT);
  double* wd = (double*)(base + OFF_WD);
  Geo<T>* geo = (Geo<T>*)(base + OFF_GEO);
  T* iw = (T*)(base + OFF_IW);
  T* K = (T*)(base + OFF_K);

  // clear what must start at zero; the previous call's contents stay otherwise
  GH_CK(cudaMemsetAsync(scal, 0, SCAL_ALLOC * sizeof(double), st));
  GH_CK(cudaMemsetAsync(status, 0, sizeof(unsigned), st));
  for (int q = 0; q < ndim; ++q) {
    GH_CK(cudaMemcpyAsync(wd + (size_t)q * NOALLOC_MAX_N, d->widths[q], (size_t)n[q] * sizeof(double),
                          cudaMemcpyHostToDevice, st));
    noalloc_geometry_kernel<T><<<(n[q] + 4 + 127) / 128, 128, 0, st>>>(n[q], lo[q], hi[q], d->theta,
                                                                       wd + (size_t)q * NOALLOC_MAX_N,
                                                                       geo + q * GEO_N, iw + q * GEO_N);
    GH_CK(cudaGetLastError());
  }

  StageArgs<T> A;
  memset(&A, 0, sizeof(A));
  for (int q = 0; q < 3; ++q) {
    const int qq = q < ndim ? q : 0;  // inactive axes are never read; point them at axis 0
    A.n[q] = n[q];
    A.bc_lo[q] = lo[q];
    A.bc_hi[q] = hi[q];
    A.geo[q] = geo + qq * GEO_N;
    A.iw[q] = iw + qq * GEO_N;
    A.wd[q] = wd + (size_t)qq * NOALLOC_MAX_N;
  }
  A.gamma = (T)d->gamma;
  A.gm1 = (T)(d->gamma - 1.0);
  A.un = uin;
  A.k1 = K;
  A.dt = scal + SCAL_DT;
  A.kchunk = kchunk;
  A.part_speed = speed;
  A.part_tot = tot;
  A.status = status;
  A.want_totals = 0;
  const dim3 grid(gx, gy, gz), block(v1.threads);

  StageArgs<T> a1 = A;
  a1.out = K;
  void* p1[] = {&a1};
  GH_CK(cudaLaunchKernel(v1.fn, grid, block, p1, v1.smem, st));
  FinalizeArgs F;
  memset(&F, 0, sizeof(F));
  F.part_speed = speed;
  F.part_tot = nullptr;
  F.nblk = (int)nblk;
  F.nv = (int)nv;
  F.mode = FIN_FIXED;
  F.fixed_dt = dt;
  F.t_end = 0.0;
  F.scal = scal;
  F.status = status;
  GH_CK(launch_finalize(F, st));
  StageArgs<T> a2 = A;
  a2.out = uout;
  void* p2[] = {&a2};
  GH_CK(cudaLaunchKernel(v2.fn, grid, block, p2, v2.smem, st));

  unsigned hs = 0;
  GH_CK(cudaMemcpyAsync(&hs, status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  GH_CK(cudaStreamSynchronize(st));
  if (hs & STATUS_NONPHYS) return fail(GENASIS_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or NaN) on the device");
  return GENASIS_OK;
}

}  // namespace gh

using namespace gh;

extern "C" int genasis_hydro_step_noalloc(const genasis_hydro_desc* d, const void* U_in, void* U_out, double dt) {
  if (!d || !U_in || !U_out) return fail(GENASIS_EINVAL, "step_noalloc: NULL argument");
  {
    // the step copies the widths from pageable memory and synchronises the
    // stream, neither of which a capturing stream allows
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    GH_CK(cudaStreamIsCapturing((cudaStream_t)d->stream, &cap));
    if (cap != cudaStreamCaptureStatusNone)
      return fail(GENASIS_EINVAL, "step_noalloc: the stream is capturing; this call synchronises and cannot be captured");
  }
  if (d->ndim < 1 || d->ndim > 3) return fail(GENASIS_EINVAL, "step_noalloc: ndim must be 1, 2 or 3");
  if (d->precision != GENASIS_FP64 && d->precision != GENASIS_FP32_MIXED)
    return fail(GENASIS_EINVAL, "step_noalloc: bad precision");
  if (d->solver != GENASIS_HLL && d->solver != GENASIS_HLLC) return fail(GENASIS_EINVAL, "step_noalloc: bad solver");
  if (!(d->gamma > 1.0) || !isfinite(d->gamma)) return fail(GENASIS_EINVAL, "step_noalloc: gamma must be > 1");
  if (!(d->theta >= 1.0 && d->theta <= 2.0)) return fail(GENASIS_EINVAL, "step_noalloc: theta must lie in [1, 2]");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(GENASIS_EINVAL, "step_noalloc: dt must be positive and finite");
  size_t ncell = 1;
  for (int q = 0; q < d->ndim; ++q) {
    if (d->n[q] < 2 || d->n[q] > NOALLOC_MAX_N)
      return fail(GENASIS_EINVAL, "step_noalloc: n[%d] = %d outside [2, %d]", q, d->n[q], NOALLOC_MAX_N);
    if (!d->widths[q]) return fail(GENASIS_EINVAL, "step_noalloc: widths[%d] is NULL", q);
    for (int i = 0; i < d->n[q]; ++i)
      if (!(d->widths[q][i] > 0.0) || !isfinite(d->widths[q][i]))
        return fail(GENASIS_EINVAL, "step_noalloc: widths[%d][%d] is not a positive finite width", q, i);
    for (int s = 0; s < 2; ++s) {
      const int bc = s ? d->bc_hi[q] : d->bc_lo[q];
      if (bc < 0 || bc > 2) return fail(GENASIS_EINVAL, "step_noalloc: bad boundary code on axis %d", q);
    }
    if ((d->bc_lo[q] == GENASIS_BC_PERIODIC) != (d->bc_hi[q] == GENASIS_BC_PERIODIC))
      return fail(GENASIS_EINVAL, "step_noalloc: axis %d: periodic must be set on both ends", q);
    ncell *= (size_t)d->n[q];
  }
  if (!is_device_ptr(U_in) || !is_device_ptr(U_out))
    return fail(GENASIS_EINVAL, "step_noalloc: U_in and U_out must be device pointers");
  const size_t bytes = ncell * (size_t)(d->ndim + 2) * (d->precision == GENASIS_FP64 ? 8 : 4);
  const char* a = (const char*)U_in;
  const char* b = (const char*)U_out;
  if (a < b + bytes && b < a + bytes) return fail(GENASIS_EINVAL, "step_noalloc: U_in and U_out overlap");
  cudaStream_t st = (cudaStream_t)d->stream;
  unsigned char* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  return d->precision == GENASIS_FP64 ? noalloc_step_t<double>(d, base, (const double*)U_in, (double*)U_out, dt, st)
                                      : noalloc_step_t<float>(d, base, (const float*)U_in, (float*)U_out, dt, st);
}
