// hydro_handle.h -- the single-mesh handle behind genasis_hydro_t, shared by
// api.cu and the multilevel driver (fmr.cu).  Internal: not part of the C ABI.
#pragma once

#include <cuda.h>
#include <string.h>

#include <type_traits>
#include <vector>

#include "aux_kernels.h"
#include "registry.h"
#include "stage_kernel.cuh"

struct genasis_hydro {
  int ndim = 0, nv = 0, n[3] = {1, 1, 1}, bc_lo[3] = {0, 0, 0}, bc_hi[3] = {0, 0, 0};
  double gamma = 1.4, theta = 1.4;
  double grad_phi[3] = {0.0, 0.0, 0.0};  // external potential gradient (source off when zero)
  int has_source = 0;
  int solver = 1, prec = 0;
  size_t ncell = 0, esize = 8;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0, num_sms = 0;
  void* U[2] = {nullptr, nullptr};
  int cur = 0;
  void* K = nullptr;
  void* geo[3] = {nullptr, nullptr, nullptr};
  void* iw[3] = {nullptr, nullptr, nullptr};
  double* wd[3] = {nullptr, nullptr, nullptr};
  float* wpair[3] = {nullptr, nullptr, nullptr};  // FP32 state: widths as hi[n] then lo[n]
  gh::dw* wdw[3] = {nullptr, nullptr, nullptr};       // double-word state: widths as pairs
  unsigned char* flags = nullptr;                 // shock bits (GENASIS_HLLC_SWITCH)
  double* part_speed = nullptr;
  double* part_tot = nullptr;
  size_t part_cap = 0;  // blocks the partial buffers hold
  double* scal = nullptr;
  unsigned* status = nullptr;
  // launch configuration
  int tile = 0, kchunk_req = 0, kchunk = 1;
  gh::StageVariant v1{}, v2{};
  dim3 grid, grid2;  // stage 1 / stage 2 (the two may use different tile shapes)
  // tensor maps of U[0], U[1] and K for TMA variants (valid when v1.tma or v2.tma)
  CUtensorMap tmap[3];
  CUtensorMap fmap[2];     // U[0], U[1] with the box of the TMA shock-flag pass
  bool flags_tma = false;  // the switch's stage-1 detector runs the TMA pass
  int want_totals = 1;
  int one_launch = 1;  // small 1D meshes: a whole advance in one cooperative launch
  int mlp_tc = 0;      // attached network: on tcgen05 (1) or mma.sync (0)
  unsigned* adv = nullptr;  // its grid-barrier words [2] (zero between launches), then one dt per CTA
  // cached graphs of `advance`, one per starting state buffer
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int g_nsteps = -1;
  double g_cfl = 0, g_tend = 0;
  // mesh as described at creation (host): low corner and widths
  double origin[3] = {0.0, 0.0, 0.0};
  std::vector<double> hw[3];
  // a batch handle (genasis_hydro_batch_create) holds only this
  genasis_batch_t batch = nullptr;
  // attached flux-correction network (genasis_hydro_set_flux_mlp): step and
  // advance run the corrected scheme of this learned solver on the state
  genasis_learned_t lf = nullptr;
};

// Single-mesh entry points refuse batch handles.
#define GH_SINGLE_MESH(h)                                                                          \
  do {                                                                                             \
    if ((h) && (h)->batch)                                                                         \
      return ::gh::fail(GENASIS_EINVAL, "%s: not a call for a batch handle (genasis_hydro_batch_*)", \
                        __func__);                                                                 \
  } while (0)

namespace gh {

// Arguments of the stage kernels for one stage of the handle's next step.
template <class T>
inline StageArgs<T> stage_args(genasis_hydro* h, int stage) {
  StageArgs<T> A;
  memset(&A, 0, sizeof(A));
  for (int q = 0; q < 3; ++q) {
    A.n[q] = h->n[q];
    A.bc_lo[q] = h->bc_lo[q];
    A.bc_hi[q] = h->bc_hi[q];
    A.geo[q] = (const Geo<T>*)h->geo[q];
    A.iw[q] = (const T*)h->iw[q];
    A.wd[q] = h->wd[q];
    if (sizeof(T) == 4) {
      const size_t nq = q < h->ndim ? (size_t)h->n[q] : 2;
      A.wdh[q] = (const T*)h->wpair[q];
      A.wdl[q] = (const T*)(h->wpair[q] + nq);
    } else if (std::is_same<T, dw>::value) {
      A.wdh[q] = (const T*)h->wdw[q];
      A.wdl[q] = (const T*)h->wdw[q];
    } else {
      A.wdh[q] = (const T*)h->wd[q];
      A.wdl[q] = (const T*)h->wd[q];
    }
  }
  A.gamma = (T)h->gamma;
  A.gm1 = (T)(h->gamma - 1.0);
  A.un = (const T*)h->U[h->cur];
  A.k1 = (const T*)h->K;
  A.out = stage == 1 ? (T*)h->K : (T*)h->U[1 - h->cur];
  A.dt = h->scal + SCAL_DT;
  A.kchunk = h->kchunk;
  A.part_speed = h->part_speed;
  A.part_tot = h->part_tot;
  A.status = h->status;
  A.want_totals = h->want_totals;
  A.has_source = h->has_source;
  A.flags = h->flags;
  for (int q = 0; q < 3; ++q) A.grad_phi[q] = (T)h->grad_phi[q];
  return A;
}

// Launch stage `stage` (1 or 2) of the handle's next step on stream st with
// its configured variant and grid (every stage launch goes through here, so
// that TMA variants get their tensor maps).
template <class T>
int launch_stage(genasis_hydro* h, int stage, cudaStream_t st);

}  // namespace gh
