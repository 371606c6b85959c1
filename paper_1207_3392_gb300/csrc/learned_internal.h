// learned_internal.h -- launchers shared between the learned-correction unit
// and the single-mesh handle (training-target support).
#pragma once

#include <cuda_runtime.h>

#include "genasis_hydro.h"
#include "learned_kernels.cuh"

namespace gh {

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
