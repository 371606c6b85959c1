// learned_internal.h -- launchers shared between the learned-correction unit
// and the single-mesh handle (training-target support).
#pragma once

#include <cuda_runtime.h>

#include "learned_kernels.cuh"

namespace gh {

cudaError_t launch_face_flux_accumulate(const Mesh2& M, int solver, const float* un, const float* k, const double* dtp,
                                        int s, double weight, double* acc, cudaStream_t st);
cudaError_t launch_restrict(int nx, int ny, int s, const float* uf, float* uc, cudaStream_t st);

}  // namespace gh
