// learned_internal.h -- launchers shared between the learned-correction unit
// and the single-mesh handle (training-target support).
#pragma once

#include <cuda_runtime.h>

#include "aux_kernels.h"
#include "genasis_hydro.h"
#include "learned_kernels.cuh"

namespace gh {

// Arguments of the one-launch corrected advance (learned_advance.cu): every
// step of a call in one cooperative launch.
struct LfAdvanceArgs {
  Mesh2 M;
  ReduceArgs<float> R;         // CFL speed: U set per step; part_speed holds one partial per CTA
  FinalizeArgs Fa;             // dt rule (mode, cfl, fixed_dt, t_end), scal, status; nblk = the grid
  float* U[2];                 // U[0]: the state at launch; step s writes U[(s + 1) & 1]
  float* K;                    // stage-1 update
  float* F;                    // plain face fluxes [nf][4]
  float* dY;                   // network outputs [nf][4]
  float* scale;                // face flux scales [nf][4]
  float* Rfct;                 // FCT ratios [ncell][8]
  unsigned char* flag[2];      // fallback flags per cell
  const mlp::InferWeights* W;  // BF16 network image, or null: the plain scheme
  int fct;                     // FCT limiting of the correction
  float ylim;                  // bound on the network outputs
  unsigned long long* nfallback;
  unsigned* status;
  unsigned* sync;              // [0..1] grid barrier, [2..3] / [4..5] all-plain flags of stage 1 / 2,
                               // [8..11] two 64-bit speed maxima; the first 48 bytes zero at launch
  double* dts;                 // one per CTA
  int nsteps;
  int mlp_tc;                  // network on tcgen05 (1) or mma.sync (0)
};

// CTA shape of the one-launch advance per network engine (measured at 256^2:
// the mma.sync network runs best as 4 CTAs of 128 threads per SM, 80 us a
// step against 82 us for 2 of 256 and 88 us for 1 of 512; the tcgen05 one as
// 1 CTA of 512 threads, four MMA groups sharing the SM's TMEM).
constexpr int lf_advance_ctas_per_sm(bool mlp_tc) { return mlp_tc ? 1 : 4; }
constexpr int lf_advance_threads(bool mlp_tc) { return 512 / lf_advance_ctas_per_sm(mlp_tc); }
// Largest cooperative grid of the one-launch advance (CTAs that fit on the
// device at once), 0 if none.
int learned_advance_max_grid(int solver, bool mlp_tc);
// Launch it with grid CTAs (1 <= grid <= learned_advance_max_grid for P.mlp_tc).
cudaError_t launch_learned_advance(const LfAdvanceArgs& P, int solver, int grid, cudaStream_t st);

cudaError_t launch_face_flux_accumulate(const Mesh2& M, int solver, const float* un, const float* k, const double* dtp,
                                        int s, double weight, double* acc, cudaStream_t st);
cudaError_t launch_restrict(int nx, int ny, int s, const float* uf, float* uc, cudaStream_t st);

// Run the corrected scheme of l on a single-mesh handle's FP32 state U and
// time *t (device pointers, same stream as l): copy them in, take nsteps CFL
// steps (nsteps > 0) or one step of dt_fixed (nsteps = 0), copy them back
// and OR l's non-physical status into *status.  Asynchronous.
int learned_run_on(genasis_learned_t l, void* U, double* t, unsigned* status, int nsteps, double cfl, double t_end,
                   double dt_fixed);

}  // namespace gh
