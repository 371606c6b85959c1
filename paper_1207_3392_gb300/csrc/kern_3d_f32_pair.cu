// kern_3d_f32_pair.cu -- 3D FP32 stage kernels that take two march planes per
// thread on the packed FP32 instructions (stage_pair.cuh).
#include "instantiate.cuh"
#include "stage_pair.cuh"

namespace gh {

namespace {

template <int SOLVER, int STAGE, int TX, int TY, int MINB>
void fill_pair(StageVariant* out) {
  using K = StagePair<SOLVER, STAGE, TX, TY>;
  out->fn = reinterpret_cast<const void*>(&hydro_stage_pair_kernel<SOLVER, STAGE, TX, TY, MINB>);
  out->smem = sizeof(typename K::Smem);
  out->tx = TX;
  out->ty = TY;
  out->threads = TX * TY;
  out->pair = 1;
}

template <int TX, int TY, int MINB>
bool pick_pair(int solver, int stage, StageVariant* out) {
  if (solver == SOLVER_HLL && stage == 1) fill_pair<SOLVER_HLL, 1, TX, TY, MINB>(out);
  else if (solver == SOLVER_HLL && stage == 2) fill_pair<SOLVER_HLL, 2, TX, TY, MINB>(out);
  else if (solver == SOLVER_HLLC && stage == 1) fill_pair<SOLVER_HLLC, 1, TX, TY, MINB>(out);
  else if (solver == SOLVER_HLLC && stage == 2) fill_pair<SOLVER_HLLC, 2, TX, TY, MINB>(out);
  else return false;
  return true;
}

}  // namespace

// Tile 11: 32 x 4 cells (x 2 planes), 3 CTAs per SM; tile 12: 32 x 7 at 2
// CTAs per SM; tile 13: 32 x 8 at 2 CTAs per SM.
bool stage_variant_3d_f32_pair(int solver, int stage, int tile, StageVariant* out) {
  switch (tile) {
    case 11: return pick_pair<32, 4, 3>(solver, stage, out);
    case 12: return pick_pair<32, 7, 2>(solver, stage, out);
    case 13: return pick_pair<32, 8, 2>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
