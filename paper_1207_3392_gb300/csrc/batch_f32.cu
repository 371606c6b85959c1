// batch_f32.cu -- persistent batch-kernel instantiations (float state).
#include "batch_kernel.cuh"
#include "batch_registry.h"

namespace gh {

template <int SOLVER, int STAGE, int TX>
static void fill(BatchVariant* out) {
  out->fn = reinterpret_cast<const void*>(&hydro_batch_kernel<float, SOLVER, STAGE, TX>);
  out->smem = BatchKernel<float, SOLVER, STAGE, TX>::SMEM;
  out->tx = TX;
  out->cols = BatchKernel<float, SOLVER, STAGE, TX>::K2::OWN;
}

template <int TX>
static bool pick(int solver, int stage, BatchVariant* out) {
  if (solver == SOLVER_HLL && stage == 1) fill<SOLVER_HLL, 1, TX>(out);
  else if (solver == SOLVER_HLL && stage == 2) fill<SOLVER_HLL, 2, TX>(out);
  else if (solver == SOLVER_HLLC && stage == 1) fill<SOLVER_HLLC, 1, TX>(out);
  else if (solver == SOLVER_HLLC && stage == 2) fill<SOLVER_HLLC, 2, TX>(out);
  else return false;
  return true;
}

bool batch_variant_f32(int solver, int stage, int tile, BatchVariant* out) {
  switch (tile) {
    case 0: return pick<128>(solver, stage, out);
    case 1: return pick<256>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
