// instantiate.cuh -- helpers that register explicit instantiations of the stage
// kernel in the variant table (one translation unit per dimensionality and
// precision so that they compile in parallel).
#pragma once

#include "registry.h"
#include "stage_kernel.cuh"

namespace gh {

template <int NDIM, class T, int SOLVER, int STAGE, int TX, int TY, int MINB, bool PRE>
inline void fill_variant(StageVariant* out) {
  using K = StageKernel<NDIM, T, SOLVER, STAGE, TX, TY, PRE>;
  out->fn = reinterpret_cast<const void*>(&hydro_stage_kernel<NDIM, T, SOLVER, STAGE, TX, TY, MINB, PRE>);
  out->smem = sizeof(typename K::Smem);
  out->tx = K::OWN;  // columns of cells per tile (TX - 1 in 1D/2D)
  out->ty = TY;
  out->threads = TX * TY;
}

// PRE: in-plane face states formed once per cell (see stage_kernel.cuh).
template <int NDIM, class T, int TX, int TY, int MINB = 1, bool PRE = (NDIM == 3)>
inline bool pick_variant(int solver, int stage, StageVariant* out) {
  if (solver == SOLVER_HLL && stage == 1) fill_variant<NDIM, T, SOLVER_HLL, 1, TX, TY, MINB, PRE>(out);
  else if (solver == SOLVER_HLL && stage == 2) fill_variant<NDIM, T, SOLVER_HLL, 2, TX, TY, MINB, PRE>(out);
  else if (solver == SOLVER_HLLC && stage == 1) fill_variant<NDIM, T, SOLVER_HLLC, 1, TX, TY, MINB, PRE>(out);
  else if (solver == SOLVER_HLLC && stage == 2) fill_variant<NDIM, T, SOLVER_HLLC, 2, TX, TY, MINB, PRE>(out);
  else return false;
  return true;
}

// HLLC with the shock switch (compiled for one tile per dimensionality).
template <int NDIM, class T, int TX, int TY, int MINB = 1, bool PRE = (NDIM == 3)>
inline bool pick_switch(int stage, StageVariant* out) {
  if (stage == 1) fill_variant<NDIM, T, SOLVER_HLLC_SW, 1, TX, TY, MINB, PRE>(out);
  else if (stage == 2) fill_variant<NDIM, T, SOLVER_HLLC_SW, 2, TX, TY, MINB, PRE>(out);
  else return false;
  return true;
}

}  // namespace gh
