// api.cu -- host runtime behind include/genasis_hydro.h: handle lifetime,
// device memory, geometry tables, launch configuration, CUDA-graph capture of
// multi-step advances, and the tile autotuner.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>
#include <type_traits>
#include <vector>

#include "genasis_hydro.h"
#include "common.h"
#include "geometry.h"
#include "aux_kernels.h"
#include "learned_internal.h"
#include "hydro_device.cuh"
#include "registry.h"
#include "stage_kernel.cuh"
#include "stage_tma.cuh"
#include "hydro_handle.h"

namespace gh {

static thread_local char g_err[512] = "no error";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int tile_count(int ndim, int prec) {
  if (prec == GENASIS_FP64_DW) return tile_count_dw(ndim);
  const bool fp64 = prec == GENASIS_FP64;
  return ndim == 1 ? tile_count_1d() : ndim == 2 ? tile_count_2d() : fp64 ? tile_count_3d_f64() : tile_count_3d_f32();
}

bool stage_variant(int ndim, int prec, int solver, int stage, int tile, StageVariant* out) {
  if (prec == GENASIS_FP64_DW) return stage_variant_dw(ndim, solver, stage, tile, out);
  const bool fp64 = prec == GENASIS_FP64;
  if (ndim == 1) return stage_variant_1d(fp64, solver, stage, tile, out);
  if (ndim == 2) return stage_variant_2d(fp64, solver, stage, tile, out);
  return fp64 ? stage_variant_3d_f64(solver, stage, tile, out) : stage_variant_3d_f32(solver, stage, tile, out);
}

int stage_tile_count(int ndim, int prec) { return tile_count(ndim, prec); }

}  // namespace gh

using namespace gh;


namespace {

int validate(const genasis_hydro_desc* d) {
  if (!d) return fail(GENASIS_EINVAL, "desc is NULL");
  if (d->ndim < 1 || d->ndim > 3) return fail(GENASIS_EINVAL, "ndim must be 1, 2 or 3 (got %d)", d->ndim);
  for (int q = 0; q < d->ndim; ++q) {
    if (d->n[q] < 2) return fail(GENASIS_EINVAL, "n[%d] = %d: need at least 2 cells", q, d->n[q]);
    if (!d->widths[q]) return fail(GENASIS_EINVAL, "widths[%d] is NULL", q);
    for (int i = 0; i < d->n[q]; ++i)
      if (!(d->widths[q][i] > 0.0) || !isfinite(d->widths[q][i]))
        return fail(GENASIS_EINVAL, "widths[%d][%d] = %g is not a positive finite width", q, i, d->widths[q][i]);
    for (int s = 0; s < 2; ++s) {
      int bc = s ? d->bc_hi[q] : d->bc_lo[q];
      if (bc < 0 || bc > 2) return fail(GENASIS_EINVAL, "bad boundary code %d on axis %d", bc, q);
    }
    if ((d->bc_lo[q] == GENASIS_BC_PERIODIC) != (d->bc_hi[q] == GENASIS_BC_PERIODIC))
      return fail(GENASIS_EINVAL, "axis %d: periodic must be set on both ends", q);
  }
  if (!(d->gamma > 1.0) || !isfinite(d->gamma)) return fail(GENASIS_EINVAL, "gamma must be > 1");
  if (d->solver != GENASIS_HLL && d->solver != GENASIS_HLLC && d->solver != GENASIS_HLLC_SWITCH)
    return fail(GENASIS_EINVAL, "bad solver %d", d->solver);
  if (d->solver == GENASIS_HLLC_SWITCH && d->precision == GENASIS_FP64_DW)
    return fail(GENASIS_EINVAL, "the shock switch is compiled for GENASIS_FP64 and GENASIS_FP32_MIXED");
  if (!(d->theta >= 1.0 && d->theta <= 2.0)) return fail(GENASIS_EINVAL, "theta must lie in [1, 2]");
  if (d->precision != GENASIS_FP64 && d->precision != GENASIS_FP32_MIXED && d->precision != GENASIS_FP64_DW)
    return fail(GENASIS_EINVAL, "bad precision %d", d->precision);
  size_t cells = 1;
  for (int q = 0; q < d->ndim; ++q) {
    cells *= (size_t)d->n[q];
    if (cells > ((size_t)1 << 34)) return fail(GENASIS_EINVAL, "mesh too large");
  }
  return GENASIS_OK;
}

template <class T>
int upload_geometry(genasis_hydro* h, const genasis_hydro_desc* d) {
  for (int q = 0; q < 3; ++q) {
    std::vector<double> w;
    if (q < h->ndim) w.assign(d->widths[q], d->widths[q] + d->n[q]);
    else w.assign(2, 1.0);  // inactive axis: unit width, never read as a flux axis
    const int n = q < h->ndim ? d->n[q] : 1;
    std::vector<double> e = extended_widths(w.data(), n < 2 ? 2 : n, h->bc_lo[q], h->bc_hi[q]);
    std::vector<Geo<T>> geo;
    std::vector<T> iw;
    append_geometry<T>(e, h->theta, geo, iw);
    GH_CK(cudaMalloc(&h->geo[q], geo.size() * sizeof(Geo<T>)));
    GH_CK(cudaMalloc(&h->iw[q], iw.size() * sizeof(T)));
    GH_CK(cudaMalloc(&h->wd[q], w.size() * sizeof(double)));
    GH_CK(cudaMemcpy(h->geo[q], geo.data(), geo.size() * sizeof(Geo<T>), cudaMemcpyHostToDevice));
    GH_CK(cudaMemcpy(h->iw[q], iw.data(), iw.size() * sizeof(T), cudaMemcpyHostToDevice));
    GH_CK(cudaMemcpy(h->wd[q], w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (sizeof(T) == 4) {
      // each FP64 width as a float pair hi + lo (for the compensated column sums)
      std::vector<float> pair(2 * w.size());
      for (size_t i = 0; i < w.size(); ++i) {
        pair[i] = (float)w[i];
        pair[w.size() + i] = (float)(w[i] - (double)pair[i]);
      }
      GH_CK(cudaMalloc(&h->wpair[q], pair.size() * sizeof(float)));
      GH_CK(cudaMemcpy(h->wpair[q], pair.data(), pair.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (std::is_same<T, dw>::value) {
      std::vector<dw> pw(w.begin(), w.end());
      GH_CK(cudaMalloc(&h->wdw[q], pw.size() * sizeof(dw)));
      GH_CK(cudaMemcpy(h->wdw[q], pw.data(), pw.size() * sizeof(dw), cudaMemcpyHostToDevice));
    }
  }
  return GENASIS_OK;
}

// A TMA variant stages 4D boxes of the FP32 state: its rows must start on
// 16-byte boundaries, so n[0] must be a multiple of 4.
bool tma_usable(const genasis_hydro* h) { return h->ndim == 3 && h->prec == GENASIS_FP32_MIXED && h->n[0] % 4 == 0; }

// Tensor map of one FP32 state array [5][n2][n1][n0] as a 4D tensor (x, y,
// z, variable) with the box of one plane of a TMA tile.
int encode_state_map(CUtensorMap* m, void* base, const int* n, int box_x, int box_y) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    GH_CK(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !fn) return fail(GENASIS_ECUDA, "cuTensorMapEncodeTiled not available");
    encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  const cuuint64_t dims[4] = {(cuuint64_t)n[0], (cuuint64_t)n[1], (cuuint64_t)n[2], 5};
  const cuuint64_t strides[3] = {(cuuint64_t)n[0] * 4, (cuuint64_t)n[0] * n[1] * 4, (cuuint64_t)n[0] * n[1] * n[2] * 4};
  const cuuint32_t box[4] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 1, 5};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(GENASIS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return GENASIS_OK;
}

int configure(genasis_hydro* h, int tile, int kchunk_req) {
  if (tile < 0 || tile >= tile_count(h->ndim, h->prec)) return fail(GENASIS_EINVAL, "tile %d out of range", tile);
  StageVariant v1, v2;
  if (!stage_variant(h->ndim, h->prec, h->solver, 1, tile, &v1) ||
      !stage_variant(h->ndim, h->prec, h->solver, 2, tile, &v2))
    return fail(GENASIS_EINVAL, "no compiled kernel for this configuration");
  if ((v1.tma || v2.tma) && !tma_usable(h))
    return fail(GENASIS_EINVAL, "tile %d stages the state with TMA, which needs a 3D FP32 mesh with n[0] a multiple of 4",
                tile);
  const int gx = (h->n[0] + v1.tx - 1) / v1.tx;
  const int gy = h->ndim == 3 ? (h->n[1] + v1.ty - 1) / v1.ty : 1;
  const int gx2 = (h->n[0] + v2.tx - 1) / v2.tx;
  const int gy2 = h->ndim == 3 ? (h->n[1] + v2.ty - 1) / v2.ty : 1;
  const int nm = h->ndim >= 2 ? h->n[h->ndim - 1] : 1;
  int kchunk = 1, gz = 1;
  if (h->ndim >= 2) {
    if (kchunk_req > 0) {
      kchunk = kchunk_req;
    } else {
      // about four CTAs per SM per stage, at least 8 planes per CTA
      const long target = 4L * h->num_sms;
      long chunks = (target + (long)gx * gy - 1) / ((long)gx * gy);
      long maxchunks = nm / 8 > 0 ? nm / 8 : 1;
      if (chunks > maxchunks) chunks = maxchunks;
      if (chunks < 1) chunks = 1;
      kchunk = (int)((nm + chunks - 1) / chunks);
    }
    if (kchunk > nm) kchunk = nm;
    if ((v1.pair || v2.pair) && (kchunk & 1)) ++kchunk;  // whole plane pairs per chunk
    gz = (nm + kchunk - 1) / kchunk;
  }
  const size_t nblk = (size_t)gx * gy * gz;
  for (const StageVariant* v : {&v1, &v2}) {
    if (v->smem > 48 * 1024) {
      GH_CK(cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v->smem));
    }
  }
  const size_t need = nblk > 4096 ? nblk : 4096;
  if (need > h->part_cap) {
    if (h->part_speed) cudaFree(h->part_speed);
    if (h->part_tot) cudaFree(h->part_tot);
    h->part_speed = nullptr;
    h->part_tot = nullptr;
    GH_CK(cudaMalloc(&h->part_speed, need * sizeof(double)));
    GH_CK(cudaMalloc(&h->part_tot, need * 5 * sizeof(double)));
    h->part_cap = need;
  }
  h->v1 = v1;
  h->v2 = v2;
  h->tile = tile;
  h->kchunk_req = kchunk_req;
  h->kchunk = kchunk;
  h->grid = dim3(gx, gy, gz);
  h->grid2 = dim3(gx2, gy2, gz);
  void* bufs[3] = {h->U[0], h->U[1], h->K};
  const StageVariant* vt = v1.tma ? &v1 : (v2.tma ? &v2 : nullptr);
  if (vt) {
    for (int i = 0; i < 3; ++i) {
      const int rc = encode_state_map(&h->tmap[i], bufs[i], h->n, vt->box_x, vt->box_y);
      if (rc) return rc;
    }
  }
  h->flags_tma = h->solver == GENASIS_HLLC_SWITCH && flags_tma_usable(h->ndim, h->prec == GENASIS_FP32_MIXED, h->n);
  if (h->flags_tma) {  // stage 1 reads U^n: maps of the two state buffers
    for (int i = 0; i < 2; ++i) {
      const int rc = encode_state_map(&h->fmap[i], bufs[i], h->n, FLAGS_TMA_BOX_X, FLAGS_TMA_BOX_Y);
      if (rc) return rc;
    }
  }
  for (int b = 0; b < 2; ++b)
    if (h->graph[b]) {
      cudaGraphExecDestroy(h->graph[b]);
      h->graph[b] = nullptr;
    }
  return GENASIS_OK;
}


template <class T>
int enqueue_flags(genasis_hydro* h, int stage) {
  if constexpr (!std::is_same<T, dw>::value) {
    if (h->solver != GENASIS_HLLC_SWITCH) return GENASIS_OK;
    FlagArgs<T> F;
    memset(&F, 0, sizeof(F));
    for (int q = 0; q < 3; ++q) {
      F.n[q] = h->n[q];
      F.bc_lo[q] = h->bc_lo[q];
      F.bc_hi[q] = h->bc_hi[q];
    }
    F.gamma = h->gamma;
    F.un = (const T*)h->U[h->cur];
    F.k1 = (const T*)h->K;
    F.dt = h->scal + SCAL_DT;
    F.flags = h->flags;
    F.ncell = h->ncell;
    F.stage = stage;
    F.status = h->status;
    if constexpr (std::is_same<T, float>::value) {
      if (h->flags_tma && stage == 1) {
        GH_CK(launch_shock_flags_tma(F, h->fmap[h->cur], h->stream));
        return GENASIS_OK;
      }
    }
    GH_CK(launch_shock_flags<T>(h->ndim, F, h->stream));
  }
  return GENASIS_OK;
}

}  // namespace

namespace gh {

template <class T>
int launch_stage(genasis_hydro* h, int stage, cudaStream_t st) {
  const StageVariant& v = stage == 1 ? h->v1 : h->v2;
  const dim3 grid = stage == 1 ? h->grid : h->grid2;
  if constexpr (std::is_same<T, float>::value) {
    if (v.tma) {
      TmaStageArgs P;
      P.A = stage_args<float>(h, stage);
      P.map_u = h->tmap[h->cur];
      P.map_k = h->tmap[2];
      void* p[] = {&P};
      GH_CK(cudaLaunchKernel(v.fn, grid, dim3(v.threads), p, v.smem, st));
      return GENASIS_OK;
    }
  }
  StageArgs<T> A = stage_args<T>(h, stage);
  void* p[] = {&A};
  GH_CK(cudaLaunchKernel(v.fn, grid, dim3(v.threads), p, v.smem, st));
  return GENASIS_OK;
}
template int launch_stage<double>(genasis_hydro*, int, cudaStream_t);
template int launch_stage<float>(genasis_hydro*, int, cudaStream_t);
template int launch_stage<dw>(genasis_hydro*, int, cudaStream_t);

}  // namespace gh

namespace {

// Small 1D meshes: every step of a call in one cooperative launch of one CTA
// per tile (kern_1d_advance.cu): 32 threads (31 cells) per CTA in FP64, so
// the FP64 work spreads over as many SMs as possible (an SM retires ~2 FP64
// operations per clock), 256 (255 cells) in FP32.
constexpr int ADV1D_MAX_CELLS = 4088;
constexpr size_t ADV1D_BYTES = 2048;  // 2 barrier words, then (at 256 B) one double per CTA

bool use_1d_advance(const genasis_hydro* h) {
  return h->one_launch && h->ndim == 1 && (h->prec == GENASIS_FP64 || h->prec == GENASIS_FP32_MIXED) &&
         (h->solver == GENASIS_HLL || h->solver == GENASIS_HLLC) && h->n[0] <= ADV1D_MAX_CELLS;
}

template <class T>
int launch_1d_advance_t(genasis_hydro* h, int nsteps, int mode, double cfl, double fixed_dt, double t_end) {
  const int tx = sizeof(T) == 8 ? 32 : 256;
  size_t smem = 0;
  const void* fn = advance_1d_kernel(sizeof(T) == 8, h->solver, tx, &smem);
  if (!fn) return fail(GENASIS_EINVAL, "no compiled one-launch kernel for this configuration");
  if (smem > 48 * 1024) GH_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  if (!h->adv) GH_CK(cudaMalloc(&h->adv, ADV1D_BYTES));
  // barrier words start at zero in every launch (even after one that gave up)
  GH_CK(cudaMemsetAsync(h->adv, 0, 2 * sizeof(unsigned), h->stream));
  StageArgs<T> A = stage_args<T>(h, 1);
  A.k1 = (const T*)h->K;
  A.kchunk = 1;
  const int ntiles = (h->n[0] + tx - 2) / (tx - 1);
  if ((size_t)ntiles * sizeof(double) > ADV1D_BYTES - 256) return fail(GENASIS_EINVAL, "mesh too large for one launch");
  FinalizeArgs F;
  memset(&F, 0, sizeof(F));
  F.part_speed = h->part_speed;
  F.part_tot = h->want_totals ? h->part_tot : nullptr;
  F.nblk = ntiles;
  F.nv = h->nv;
  F.mode = mode;
  F.cfl = cfl;
  F.fixed_dt = fixed_dt;
  F.t_end = t_end;
  F.scal = h->scal;
  F.status = h->status;
  T* ua = (T*)h->U[h->cur];
  T* ub = (T*)h->U[1 - h->cur];
  unsigned* bar = h->adv;
  double* dts = (double*)((char*)h->adv + 256);
  void* args[] = {&A, &F, &nsteps, &ua, &ub, &bar, &dts};
  // cooperative: the CTAs wait on one another, so all must be resident
  GH_CK(cudaLaunchCooperativeKernel(fn, dim3(ntiles), dim3(tx), args, smem, h->stream));
  h->cur ^= nsteps & 1;
  return GENASIS_OK;
}

int launch_1d_advance(genasis_hydro* h, int nsteps, int mode, double cfl, double fixed_dt, double t_end) {
  return h->prec == GENASIS_FP64 ? launch_1d_advance_t<double>(h, nsteps, mode, cfl, fixed_dt, t_end)
                                 : launch_1d_advance_t<float>(h, nsteps, mode, cfl, fixed_dt, t_end);
}

template <class T>
int enqueue_step_t(genasis_hydro* h, int mode, double fixed_dt, double cfl, double t_end, cudaEvent_t* ev) {
  if (ev) GH_CK(cudaEventRecord(ev[0], h->stream));
  int rc = enqueue_flags<T>(h, 1);
  if (rc) return rc;
  rc = launch_stage<T>(h, 1, h->stream);
  if (rc) return rc;
  if (ev) GH_CK(cudaEventRecord(ev[1], h->stream));
  FinalizeArgs F;
  F.part_speed = h->part_speed;
  F.part_tot = h->want_totals ? h->part_tot : nullptr;
  F.nblk = (int)(h->grid.x * h->grid.y * h->grid.z);
  F.nv = h->nv;
  F.mode = mode;
  F.cfl = cfl;
  F.fixed_dt = fixed_dt;
  F.t_end = t_end;
  F.scal = h->scal;
  F.status = h->status;
  GH_CK(launch_finalize(F, h->stream));
  if (ev) GH_CK(cudaEventRecord(ev[2], h->stream));
  rc = enqueue_flags<T>(h, 2);
  if (rc) return rc;
  rc = launch_stage<T>(h, 2, h->stream);
  if (rc) return rc;
  if (ev) GH_CK(cudaEventRecord(ev[3], h->stream));
  h->cur = 1 - h->cur;
  return GENASIS_OK;
}

int enqueue_step(genasis_hydro* h, int mode, double fixed_dt, double cfl, double t_end,
                 cudaEvent_t* ev = nullptr) {
  return h->prec == GENASIS_FP64         ? enqueue_step_t<double>(h, mode, fixed_dt, cfl, t_end, ev)
         : h->prec == GENASIS_FP32_MIXED ? enqueue_step_t<float>(h, mode, fixed_dt, cfl, t_end, ev)
                                         : enqueue_step_t<dw>(h, mode, fixed_dt, cfl, t_end, ev);
}

template <class T>
ReduceArgs<T> reduce_args(genasis_hydro* h) {
  ReduceArgs<T> A;
  memset(&A, 0, sizeof(A));
  A.ncell = h->ncell;
  for (int q = 0; q < 3; ++q) {
    A.n[q] = h->n[q];
    A.iw[q] = (const T*)h->iw[q];
    A.wd[q] = h->wd[q];
  }
  A.gamma = h->gamma;
  A.U = (const T*)h->U[h->cur];
  A.part_speed = h->part_speed;
  A.part_tot = h->part_tot;
  A.status = h->status;
  size_t nb = (h->ncell + 255) / 256;
  A.nblk = (int)(nb > 2048 ? 2048 : (nb < 1 ? 1 : nb));
  return A;
}

int reduce_now(genasis_hydro* h, bool speed) {
  int nblk;
  if (h->prec == GENASIS_FP64) {
    ReduceArgs<double> A = reduce_args<double>(h);
    nblk = A.nblk;
    GH_CK(speed ? launch_speed<double>(h->ndim, A, h->stream) : launch_totals<double>(h->ndim, A, h->stream));
  } else if (h->prec == GENASIS_FP32_MIXED) {
    ReduceArgs<float> A = reduce_args<float>(h);
    nblk = A.nblk;
    GH_CK(speed ? launch_speed<float>(h->ndim, A, h->stream) : launch_totals<float>(h->ndim, A, h->stream));
  } else {
    ReduceArgs<dw> A = reduce_args<dw>(h);
    nblk = A.nblk;
    GH_CK(speed ? launch_speed<dw>(h->ndim, A, h->stream) : launch_totals<dw>(h->ndim, A, h->stream));
  }
  FinalizeArgs F;
  memset(&F, 0, sizeof(F));
  F.part_speed = speed ? h->part_speed : nullptr;
  F.part_tot = speed ? nullptr : h->part_tot;
  F.nblk = nblk;
  F.nv = h->nv;
  F.mode = FIN_REDUCE;
  F.scal = h->scal;
  F.status = h->status;
  GH_CK(launch_finalize(F, h->stream));
  return GENASIS_OK;
}

int sync_status(genasis_hydro* h) {
  unsigned st = 0;
  GH_CK(cudaMemcpyAsync(&st, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  GH_CK(cudaStreamSynchronize(h->stream));
  if (st & STATUS_NONPHYS) return fail(GENASIS_ENONPHYS, "non-physical state (rho <= 0, p <= 0 or NaN) on the device");
  if (st & STATUS_TIMEOUT) return fail(GENASIS_ETIMEOUT, "a bounded device wait gave up");
  return GENASIS_OK;
}

// Copy `count` elements of precision `src_prec` from src (host or device) into
// device buffer dst of the handle's precision.
int import_array(genasis_hydro* h, const void* src, int src_prec, size_t count, void* dst) {
  const size_t ssize = src_prec == GENASIS_FP64 ? 8 : 4;
  const bool dev = is_device_ptr(src);
  if (src_prec == h->prec) {
    GH_CK(cudaMemcpyAsync(dst, src, count * ssize, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    return GENASIS_OK;
  }
  const void* dsrc = src;
  void* tmp = nullptr;
  if (!dev) {
    GH_CK(cudaMallocAsync(&tmp, count * ssize, h->stream));
    GH_CK(cudaMemcpyAsync(tmp, src, count * ssize, cudaMemcpyHostToDevice, h->stream));
    dsrc = tmp;
  }
  cudaError_t e;
  if (h->prec == GENASIS_FP64_DW)
    e = src_prec == GENASIS_FP64 ? launch_convert<double, dw>(count, (const double*)dsrc, (dw*)dst, h->stream)
                                 : launch_convert<float, dw>(count, (const float*)dsrc, (dw*)dst, h->stream);
  else
    e = src_prec == GENASIS_FP64 ? launch_convert<double, float>(count, (const double*)dsrc, (float*)dst, h->stream)
                                 : launch_convert<float, double>(count, (const float*)dsrc, (double*)dst, h->stream);
  if (tmp) cudaFreeAsync(tmp, h->stream);
  GH_CK(e);
  return GENASIS_OK;
}

// Enqueue the copy of the current state into U (host or device) in the given
// precision, converting on the device if it differs from the handle's.
int export_array(genasis_hydro* h, void* U, int precision) {
  const size_t count = h->ncell * h->nv;
  const bool dev = is_device_ptr(U);
  if (precision == h->prec) {
    GH_CK(cudaMemcpyAsync(U, h->U[h->cur], count * h->esize, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          h->stream));
    return GENASIS_OK;
  }
  const size_t dsize = precision == GENASIS_FP64 ? 8 : 4;
  void* dst = U;
  if (!dev) GH_CK(cudaMallocAsync(&dst, count * dsize, h->stream));
  const void* src = h->U[h->cur];
  cudaError_t e;
  if (h->prec == GENASIS_FP64_DW)
    e = precision == GENASIS_FP64 ? launch_convert<dw, double>(count, (const dw*)src, (double*)dst, h->stream)
                                  : launch_convert<dw, float>(count, (const dw*)src, (float*)dst, h->stream);
  else
    e = h->prec == GENASIS_FP64 ? launch_convert<double, float>(count, (const double*)src, (float*)dst, h->stream)
                                : launch_convert<float, double>(count, (const float*)src, (double*)dst, h->stream);
  GH_CK(e);
  if (!dev) {
    GH_CK(cudaMemcpyAsync(U, dst, count * dsize, cudaMemcpyDeviceToHost, h->stream));
    GH_CK(cudaFreeAsync(dst, h->stream));
  }
  return GENASIS_OK;
}

int free_all(genasis_hydro* h) {
  if (h->batch) genasis_batch_destroy(h->batch);
  cudaFree(h->adv);
  if (h->lf) genasis_learned_destroy(h->lf);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (int b = 0; b < 2; ++b)
    if (h->graph[b]) cudaGraphExecDestroy(h->graph[b]);
  for (int b = 0; b < 2; ++b) cudaFree(h->U[b]);
  cudaFree(h->K);
  for (int q = 0; q < 3; ++q) {
    cudaFree(h->geo[q]);
    cudaFree(h->iw[q]);
    cudaFree(h->wd[q]);
    cudaFree(h->wpair[q]);
    cudaFree(h->wdw[q]);
  }
  cudaFree(h->part_speed);
  cudaFree(h->part_tot);
  cudaFree(h->flags);
  cudaFree(h->scal);
  cudaFree(h->status);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return GENASIS_OK;
}

}  // namespace

extern "C" {

const char* genasis_hydro_last_error(void) { return g_err; }

int genasis_hydro_create(const genasis_hydro_desc* d, genasis_hydro_t* out) {
  if (!out) return fail(GENASIS_EINVAL, "out is NULL");
  *out = nullptr;
  int rc = validate(d);
  if (rc) return rc;
  genasis_hydro* h = new genasis_hydro();
  h->ndim = d->ndim;
  h->nv = d->ndim + 2;
  h->ncell = 1;
  for (int q = 0; q < 3; ++q) {
    h->n[q] = q < d->ndim ? d->n[q] : 1;
    h->bc_lo[q] = q < d->ndim ? d->bc_lo[q] : GENASIS_BC_OUTFLOW;
    h->bc_hi[q] = q < d->ndim ? d->bc_hi[q] : GENASIS_BC_OUTFLOW;
    h->ncell *= (size_t)h->n[q];
  }
  for (int q = 0; q < d->ndim; ++q) {
    h->origin[q] = d->origin[q];
    h->hw[q].assign(d->widths[q], d->widths[q] + d->n[q]);
  }
  h->gamma = d->gamma;
  h->theta = d->theta;
  // in 1D no face is transverse to a shock: the switch is plain HLLC
  h->solver = d->solver == GENASIS_HLLC_SWITCH && d->ndim == 1 ? GENASIS_HLLC : d->solver;
  h->prec = d->precision;
  h->esize = h->prec == GENASIS_FP32_MIXED ? 4 : 8;
#define GH_CK_CREATE(call)                                                                          \
  do {                                                                                              \
    cudaError_t e_ = (call);                                                                        \
    if (e_ != cudaSuccess) {                                                                        \
      int code_ = fail(e_ == cudaErrorMemoryAllocation ? GENASIS_ENOMEM : GENASIS_ECUDA, "%s: %s", #call, \
                       cudaGetErrorString(e_));                                                     \
      free_all(h);                                                                                  \
      return code_;                                                                                 \
    }                                                                                               \
  } while (0)
  GH_CK_CREATE(cudaGetDevice(&h->device));
  GH_CK_CREATE(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
  if (d->stream) {
    h->stream = (cudaStream_t)d->stream;
  } else {
    GH_CK_CREATE(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  const size_t bytes = h->ncell * h->nv * h->esize;
  for (int b = 0; b < 2; ++b) {
    GH_CK_CREATE(cudaMalloc(&h->U[b], bytes));
    GH_CK_CREATE(cudaMemsetAsync(h->U[b], 0, bytes, h->stream));
  }
  GH_CK_CREATE(cudaMalloc(&h->K, bytes));
  if (h->solver == GENASIS_HLLC_SWITCH) GH_CK_CREATE(cudaMalloc(&h->flags, h->ncell));
  GH_CK_CREATE(cudaMalloc(&h->scal, SCAL_ALLOC * sizeof(double)));
  GH_CK_CREATE(cudaMemsetAsync(h->scal, 0, SCAL_ALLOC * sizeof(double), h->stream));
  GH_CK_CREATE(cudaMalloc(&h->status, sizeof(unsigned)));
  GH_CK_CREATE(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
  rc = h->prec == GENASIS_FP64         ? upload_geometry<double>(h, d)
       : h->prec == GENASIS_FP32_MIXED ? upload_geometry<float>(h, d)
                                       : upload_geometry<dw>(h, d);
  if (!rc) rc = configure(h, 0, 0);
  if (rc) {
    free_all(h);
    return rc;
  }
  GH_CK_CREATE(cudaStreamSynchronize(h->stream));
#undef GH_CK_CREATE
  *out = h;
  return GENASIS_OK;
}

int genasis_hydro_destroy(genasis_hydro_t h) {
  if (!h) return GENASIS_OK;
  return free_all(h);
}

int genasis_hydro_set_primitive(genasis_hydro_t h, const double* rho, const double* vel, const double* p) {
  GH_SINGLE_MESH(h);
  if (!h || !rho || !vel || !p) return fail(GENASIS_EINVAL, "NULL argument");
  const double* src[3] = {rho, vel, p};
  const size_t cnt[3] = {h->ncell, h->ncell * h->ndim, h->ncell};
  double* dev[3] = {nullptr, nullptr, nullptr};
  int rc = GENASIS_OK;
  for (int a = 0; a < 3 && !rc; ++a) {
    if (is_device_ptr(src[a])) continue;
    cudaError_t e = cudaMallocAsync((void**)&dev[a], cnt[a] * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dev[a], src[a], cnt[a] * sizeof(double), cudaMemcpyHostToDevice, h->stream);
    if (e != cudaSuccess) rc = fail(GENASIS_ECUDA, "staging primitives: %s", cudaGetErrorString(e));
  }
  if (!rc) {
    const double* r = dev[0] ? dev[0] : rho;
    const double* v = dev[1] ? dev[1] : vel;
    const double* pp = dev[2] ? dev[2] : p;
    void* U = h->U[h->cur];
    cudaError_t e =
        h->prec == GENASIS_FP64
            ? launch_init_from_primitive<double>(h->ndim, h->ncell, h->gamma, r, v, pp, (double*)U, h->stream)
        : h->prec == GENASIS_FP32_MIXED
            ? launch_init_from_primitive<float>(h->ndim, h->ncell, h->gamma, r, v, pp, (float*)U, h->stream)
            : launch_init_from_primitive<dw>(h->ndim, h->ncell, h->gamma, r, v, pp, (dw*)U, h->stream);
    if (e != cudaSuccess) rc = fail(GENASIS_ECUDA, "init kernel: %s", cudaGetErrorString(e));
  }
  for (int a = 0; a < 3; ++a)
    if (dev[a]) cudaFreeAsync(dev[a], h->stream);
  if (!rc) {
    GH_CK(cudaMemsetAsync(h->scal + SCAL_T, 0, sizeof(double), h->stream));
    if (!is_device_ptr(rho) || !is_device_ptr(vel) || !is_device_ptr(p)) GH_CK(cudaStreamSynchronize(h->stream));
  }
  return rc;
}

int genasis_hydro_set_conserved(genasis_hydro_t h, const void* U, int precision) {
  GH_SINGLE_MESH(h);
  if (!h || !U) return fail(GENASIS_EINVAL, "NULL argument");
  if (precision != GENASIS_FP64 && precision != GENASIS_FP32_MIXED) return fail(GENASIS_EINVAL, "bad precision");
  int rc = import_array(h, U, precision, h->ncell * h->nv, h->U[h->cur]);
  if (rc) return rc;
  if (!is_device_ptr(U)) GH_CK(cudaStreamSynchronize(h->stream));
  return GENASIS_OK;
}

int genasis_hydro_set_conserved_async(genasis_hydro_t h, const void* U, int precision) {
  GH_SINGLE_MESH(h);
  if (!h || !U) return fail(GENASIS_EINVAL, "NULL argument");
  if (precision != GENASIS_FP64 && precision != GENASIS_FP32_MIXED) return fail(GENASIS_EINVAL, "bad precision");
  return import_array(h, U, precision, h->ncell * h->nv, h->U[h->cur]);
}

int genasis_hydro_get_conserved_async(genasis_hydro_t h, void* U, int precision) {
  GH_SINGLE_MESH(h);
  if (!h || !U) return fail(GENASIS_EINVAL, "NULL argument");
  if (precision != GENASIS_FP64 && precision != GENASIS_FP32_MIXED) return fail(GENASIS_EINVAL, "bad precision");
  return export_array(h, U, precision);
}

int genasis_hydro_sync(genasis_hydro_t h) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  return sync_status(h);
}

int genasis_hydro_get_conserved(genasis_hydro_t h, void* U, int precision) {
  GH_SINGLE_MESH(h);
  if (!h || !U) return fail(GENASIS_EINVAL, "NULL argument");
  if (precision != GENASIS_FP64 && precision != GENASIS_FP32_MIXED) return fail(GENASIS_EINVAL, "bad precision");
  int rc = export_array(h, U, precision);
  if (rc) return rc;
  return sync_status(h);
}


int genasis_hydro_compute_dt(genasis_hydro_t h, double cfl, double* dt) {
  GH_SINGLE_MESH(h);
  if (!h || !dt) return fail(GENASIS_EINVAL, "NULL argument");
  if (!(cfl > 0.0)) return fail(GENASIS_EINVAL, "cfl must be > 0");
  int rc = reduce_now(h, true);
  if (rc) return rc;
  double v = 0;
  GH_CK(cudaMemcpyAsync(&v, h->scal + SCAL_DTCFL, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  rc = sync_status(h);
  if (rc) return rc;
  *dt = cfl * v;
  return GENASIS_OK;
}

int genasis_hydro_step(genasis_hydro_t h, double dt) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(GENASIS_EINVAL, "dt must be positive and finite");
  if (h->lf) return learned_run_on(h->lf, h->U[h->cur], h->scal + SCAL_T, h->status, 0, 0.0, 0.0, dt);
  if (use_1d_advance(h)) return launch_1d_advance(h, 1, FIN_FIXED, 0.0, dt, 0.0);
  return enqueue_step(h, FIN_FIXED, dt, 0.0, 0.0);
}

int genasis_hydro_advance(genasis_hydro_t h, int nsteps, double cfl, double t_end, double* t_out) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  if (nsteps < 0) return fail(GENASIS_EINVAL, "nsteps < 0");
  if (!(cfl > 0.0)) return fail(GENASIS_EINVAL, "cfl must be > 0");
  if (h->lf && nsteps > 0) {
    int rc = learned_run_on(h->lf, h->U[h->cur], h->scal + SCAL_T, h->status, nsteps, cfl, t_end, 0.0);
    if (rc) return rc;
  } else if (nsteps > 0 && use_1d_advance(h)) {
    int rc = launch_1d_advance(h, nsteps, FIN_CFL, cfl, 0.0, t_end);
    if (rc) return rc;
  } else if (nsteps > 0) {
    const int cur0 = h->cur;
    if (h->g_nsteps != nsteps || h->g_cfl != cfl || h->g_tend != t_end) {
      for (int b = 0; b < 2; ++b)
        if (h->graph[b]) {
          cudaGraphExecDestroy(h->graph[b]);
          h->graph[b] = nullptr;
        }
      h->g_nsteps = nsteps;
      h->g_cfl = cfl;
      h->g_tend = t_end;
    }
    if (!h->graph[cur0]) {
      cudaGraph_t g;
      GH_CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      int rc = GENASIS_OK;
      for (int s = 0; s < nsteps && !rc; ++s) rc = enqueue_step(h, FIN_CFL, 0.0, cfl, t_end);
      cudaError_t e = cudaStreamEndCapture(h->stream, &g);
      h->cur = cur0;
      if (rc) {
        if (e == cudaSuccess) cudaGraphDestroy(g);
        return rc;
      }
      GH_CK(e);
      e = cudaGraphInstantiate(&h->graph[cur0], g, 0);
      cudaGraphDestroy(g);
      GH_CK(e);
    }
    GH_CK(cudaGraphLaunch(h->graph[cur0], h->stream));
    h->cur = cur0 ^ (nsteps & 1);
  }
  if (t_out) {
    GH_CK(cudaMemcpyAsync(t_out, h->scal + SCAL_T, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return sync_status(h);
  }
  return GENASIS_OK;
}

int genasis_hydro_get_time(genasis_hydro_t h, double* t) {
  GH_SINGLE_MESH(h);
  if (!h || !t) return fail(GENASIS_EINVAL, "NULL argument");
  GH_CK(cudaMemcpyAsync(t, h->scal + SCAL_T, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  GH_CK(cudaStreamSynchronize(h->stream));
  return GENASIS_OK;
}

int genasis_hydro_set_time(genasis_hydro_t h, double t) {
  GH_SINGLE_MESH(h);
  if (!h || !isfinite(t)) return fail(GENASIS_EINVAL, "bad argument");
  GH_CK(cudaMemcpyAsync(h->scal + SCAL_T, &t, sizeof(double), cudaMemcpyHostToDevice, h->stream));
  GH_CK(cudaStreamSynchronize(h->stream));
  return GENASIS_OK;
}

int genasis_hydro_get_totals(genasis_hydro_t h, double* totals) {
  GH_SINGLE_MESH(h);
  if (!h || !totals) return fail(GENASIS_EINVAL, "NULL argument");
  int rc = reduce_now(h, false);
  if (rc) return rc;
  GH_CK(cudaMemcpyAsync(totals, h->scal + SCAL_TOT, h->nv * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return sync_status(h);
}

int genasis_hydro_status(genasis_hydro_t h) {
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  if (h->batch) return genasis_batch_status(h->batch, nullptr);
  return sync_status(h);
}

int genasis_hydro_clear_status(genasis_hydro_t h) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  GH_CK(cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream));
  GH_CK(cudaStreamSynchronize(h->stream));
  return GENASIS_OK;
}

int genasis_hydro_set_tile(genasis_hydro_t h, int tile, int kchunk) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  if (kchunk < 0) return fail(GENASIS_EINVAL, "kchunk < 0");
  GH_CK(cudaStreamSynchronize(h->stream));
  return configure(h, tile, kchunk);
}

int genasis_hydro_get_tile(genasis_hydro_t h, int* info) {
  GH_SINGLE_MESH(h);
  if (!h || !info) return fail(GENASIS_EINVAL, "NULL argument");
  info[0] = h->tile;
  info[1] = h->v1.tx;
  info[2] = h->v1.ty;
  info[3] = h->kchunk;
  info[4] = (int)(h->grid.x * h->grid.y * h->grid.z);
  info[5] = tile_count(h->ndim, h->prec);
  return GENASIS_OK;
}

int genasis_hydro_set_option(genasis_hydro_t h, int option, int value) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  if (option == GENASIS_OPT_STEP_TOTALS) {
    if (value != 0 && value != 1) return fail(GENASIS_EINVAL, "GENASIS_OPT_STEP_TOTALS takes 0 or 1");
    if (h->want_totals != value) {
      h->want_totals = value;
      for (int b = 0; b < 2; ++b)
        if (h->graph[b]) {
          cudaGraphExecDestroy(h->graph[b]);
          h->graph[b] = nullptr;
        }
    }
    return GENASIS_OK;
  }
  if (option == GENASIS_OPT_ONE_LAUNCH) {
    if (value != 0 && value != 1) return fail(GENASIS_EINVAL, "GENASIS_OPT_ONE_LAUNCH takes 0 or 1");
    h->one_launch = value;
    if (h->lf) return genasis_learned_set_option(h->lf, option, value);
    return GENASIS_OK;
  }
  if (option == GENASIS_OPT_MLP_TCGEN05) {
    if (value != 0 && value != 1) return fail(GENASIS_EINVAL, "GENASIS_OPT_MLP_TCGEN05 takes 0 or 1");
    h->mlp_tc = value;
    if (h->lf) return genasis_learned_set_option(h->lf, option, value);
    return GENASIS_OK;
  }
  return fail(GENASIS_EINVAL, "unknown option %d", option);
}

int genasis_hydro_set_potential_gradient(genasis_hydro_t h, const double* grad_phi) {
  GH_SINGLE_MESH(h);
  if (!h || !grad_phi) return fail(GENASIS_EINVAL, "NULL argument");
  for (int q = 0; q < 3; ++q)
    if (!(fabs(grad_phi[q]) < INFINITY)) return fail(GENASIS_EINVAL, "potential gradient must be finite");
  int on = 0;
  for (int q = 0; q < 3; ++q) {
    h->grad_phi[q] = q < h->ndim ? grad_phi[q] : 0.0;
    on |= h->grad_phi[q] != 0.0;
  }
  h->has_source = on;
  for (int b = 0; b < 2; ++b)  // captured step graphs hold the old arguments
    if (h->graph[b]) {
      cudaGraphExecDestroy(h->graph[b]);
      h->graph[b] = nullptr;
    }
  return GENASIS_OK;
}

int genasis_hydro_get_step_totals(genasis_hydro_t h, double* totals) {
  GH_SINGLE_MESH(h);
  if (!h || !totals) return fail(GENASIS_EINVAL, "NULL argument");
  GH_CK(cudaMemcpyAsync(totals, h->scal + SCAL_TOT, h->nv * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return sync_status(h);
}

static int mesh2_of(genasis_hydro* h, Mesh2* M) {
  if (h->ndim != 2 || h->prec != GENASIS_FP32_MIXED)
    return fail(GENASIS_EINVAL, "needs a 2D GENASIS_FP32_MIXED handle");
  M->nx = h->n[0];
  M->ny = h->n[1];
  for (int q = 0; q < 2; ++q) {
    M->bc_lo[q] = h->bc_lo[q];
    M->bc_hi[q] = h->bc_hi[q];
    M->geo[q] = (const Geo<float>*)h->geo[q];
    M->iw[q] = (const float*)h->iw[q];
  }
  M->gamma = (float)h->gamma;
  M->gm1 = (float)(h->gamma - 1.0);
  return GENASIS_OK;
}

int genasis_hydro_accumulate_face_flux(genasis_hydro_t h, int stride, double weight, double* F) {
  GH_SINGLE_MESH(h);
  if (!h || !F) return fail(GENASIS_EINVAL, "NULL argument");
  Mesh2 M;
  int rc = mesh2_of(h, &M);
  if (rc) return rc;
  if (stride < 1 || M.nx % stride || M.ny % stride) return fail(GENASIS_EINVAL, "stride must divide nx and ny");
  if (!is_device_ptr(F)) return fail(GENASIS_EINVAL, "F must be a device pointer");
  // the last step read U^n from the other state buffer and left its K
  GH_CK(launch_face_flux_accumulate(M, h->solver, (const float*)h->U[1 - h->cur], (const float*)h->K, h->scal + SCAL_DT,
                                    stride, weight, F, h->stream));
  return GENASIS_OK;
}

int genasis_hydro_restrict(genasis_hydro_t h, int factor, float* U_coarse) {
  GH_SINGLE_MESH(h);
  if (!h || !U_coarse) return fail(GENASIS_EINVAL, "NULL argument");
  Mesh2 M;
  int rc = mesh2_of(h, &M);
  if (rc) return rc;
  if (factor < 1 || M.nx % factor || M.ny % factor) return fail(GENASIS_EINVAL, "factor must divide nx and ny");
  if (!is_device_ptr(U_coarse)) return fail(GENASIS_EINVAL, "U_coarse must be a device pointer");
  GH_CK(launch_restrict(M.nx, M.ny, factor, (const float*)h->U[h->cur], U_coarse, h->stream));
  GH_CK(cudaStreamSynchronize(h->stream));
  return GENASIS_OK;
}

int genasis_hydro_launches_per_step(genasis_hydro_t h) {
  GH_SINGLE_MESH(h);
  if (!h) return fail(GENASIS_EINVAL, "NULL handle");
  if (use_1d_advance(h)) return 1;  // one launch covers all the steps of a call
  if (h->lf) {  // the corrected scheme, and the kernel that passes its status back
    const int n = genasis_learned_launches_per_step(h->lf);
    return n < 0 ? n : n + 1;
  }
  return h->solver == GENASIS_HLLC_SWITCH ? 5 : 3;
}

int genasis_hydro_profile_step(genasis_hydro_t h, double cfl, float* ms) {
  GH_SINGLE_MESH(h);
  if (!h || !ms) return fail(GENASIS_EINVAL, "NULL argument");
  if (!(cfl > 0.0)) return fail(GENASIS_EINVAL, "cfl must be > 0");
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  int rc = GENASIS_OK;
  for (int i = 0; i < 4 && !rc; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) rc = fail(GENASIS_ECUDA, "cudaEventCreate failed");
  if (!rc) rc = enqueue_step(h, FIN_CFL, 0.0, cfl, 0.0, ev);
  if (!rc && cudaEventSynchronize(ev[3]) != cudaSuccess) rc = fail(GENASIS_ECUDA, "profile sync failed");
  if (!rc) {
    cudaEventElapsedTime(&ms[0], ev[0], ev[1]);
    cudaEventElapsedTime(&ms[1], ev[1], ev[2]);
    cudaEventElapsedTime(&ms[2], ev[2], ev[3]);
  }
  for (int i = 0; i < 4; ++i)
    if (ev[i]) cudaEventDestroy(ev[i]);
  if (rc) return rc;
  return sync_status(h);
}

int genasis_hydro_autotune(genasis_hydro_t h, int trial_steps, const char* cache_path) {
  GH_SINGLE_MESH(h);
  if (!h || trial_steps < 1) return fail(GENASIS_EINVAL, "bad argument");
  char key[160];
  snprintf(key, sizeof(key), "ndim=%d n=%d,%d,%d prec=%d solver=%d", h->ndim, h->n[0], h->n[1], h->n[2], h->prec,
           h->solver);
  if (cache_path) {
    FILE* f = fopen(cache_path, "r");
    if (f) {
      char line[256];
      int tile = -1, kc = -1;
      while (fgets(line, sizeof(line), f)) {
        const size_t kl = strlen(key);
        if (strncmp(line, key, kl) == 0 && line[kl] == ' ') {
          int t2, k2;
          if (sscanf(line + kl, " tile=%d kchunk=%d", &t2, &k2) == 2) {
            tile = t2;
            kc = k2;
          }
        }
      }
      fclose(f);
      if (tile >= 0 && tile < tile_count(h->ndim, h->prec)) return configure(h, tile, kc);
    }
  }
  // save state, time, status
  const size_t bytes = h->ncell * h->nv * h->esize;
  void* save = nullptr;
  double scal_save[SCAL_COUNT];
  GH_CK(cudaMalloc(&save, bytes));
  GH_CK(cudaMemcpyAsync(save, h->U[h->cur], bytes, cudaMemcpyDeviceToDevice, h->stream));
  GH_CK(cudaMemcpyAsync(scal_save, h->scal, sizeof(scal_save), cudaMemcpyDeviceToHost, h->stream));
  const int cur_save = h->cur;
  cudaEvent_t e0, e1;
  GH_CK(cudaEventCreate(&e0));
  GH_CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_tile = 0, best_kc = 0;
  int rc = GENASIS_OK;
  const int nm = h->ndim >= 2 ? h->n[h->ndim - 1] : 1;
  for (int tile = 0; tile < tile_count(h->ndim, h->prec) && !rc; ++tile) {
    StageVariant probe, probe2;
    if (!stage_variant(h->ndim, h->prec, h->solver, 1, tile, &probe) ||
        !stage_variant(h->ndim, h->prec, h->solver, 2, tile, &probe2))
      continue;  // not compiled for this solver
    if ((probe.tma || probe2.tma) && !tma_usable(h)) continue;  // TMA tile on an unaligned mesh
    // the paired tiles round differently (explicit roundings, not the
    // compiler's fused products): tuning keeps the bits of the default tile
    if (probe.pair || probe2.pair) continue;
    std::vector<int> kcs = {0};
    if (h->ndim == 2)  // small 2D meshes need short chunks to fill the GPU
      for (int kc : {2, 4, 8})
        if (kc < nm) kcs.push_back(kc);
    if (h->ndim >= 2)
      for (int kc : {12, 16, 24, 32, 40, 48, 64})
        if (kc < nm) kcs.push_back(kc);
    for (int kc : kcs) {
      rc = configure(h, tile, kc);
      if (rc) break;
      rc = enqueue_step(h, FIN_CFL, 0.0, 0.1, 0.0);  // warm-up
      if (rc) break;
      cudaEventRecord(e0, h->stream);
      for (int s = 0; s < trial_steps && !rc; ++s) rc = enqueue_step(h, FIN_CFL, 0.0, 0.1, 0.0);
      cudaEventRecord(e1, h->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(GENASIS_ECUDA, "autotune timing failed");
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (!rc && ms < best) {
        best = ms;
        best_tile = tile;
        best_kc = kc;
      }
      // restore the state after every trial
      h->cur = cur_save;
      cudaMemcpyAsync(h->U[h->cur], save, bytes, cudaMemcpyDeviceToDevice, h->stream);
    }
  }
  cudaMemcpyAsync(h->scal, scal_save, sizeof(scal_save), cudaMemcpyHostToDevice, h->stream);
  cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream);
  cudaStreamSynchronize(h->stream);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  rc = configure(h, best_tile, best_kc);
  if (rc) return rc;
  if (cache_path) {
    FILE* f = fopen(cache_path, "a");
    if (f) {
      fprintf(f, "%s tile=%d kchunk=%d ms_per_step=%.6f\n", key, best_tile, best_kc, best / trial_steps);
      fclose(f);
    }
  }
  return GENASIS_OK;
}

}  // extern "C"
