// kern_3d_f32_tma.cu -- 3D FP32 stage kernels whose state planes are staged
// in shared memory by TMA (stage_tma.cuh).
#include "instantiate.cuh"
#include "stage_tma.cuh"

namespace gh {

namespace {

template <int SOLVER, int STAGE, int TX, int TY, int NS, int MINB>
void fill_tma(StageVariant* out) {
  using K = StageTma<SOLVER, STAGE, TX, TY, NS>;
  out->fn = reinterpret_cast<const void*>(&hydro_stage_tma_kernel<SOLVER, STAGE, TX, TY, NS, MINB>);
  out->smem = sizeof(typename K::Smem);
  out->tx = TX;
  out->ty = TY;
  out->threads = K::NTHR;
  out->tma = 1;
  out->box_x = K::XB;
  out->box_y = K::YB;
}

// Stage 1 staged by TMA (tile 9: 32 x 6 cells + the producer warp, 3 slots,
// 4 CTAs per SM; tile 10: 32 x 8 at 3 CTAs per SM); stage 2 the 32 x 7
// kernel of tile 8.
template <int SOLVER>
bool pick_tma(int tile, int stage, StageVariant* out) {
  if (stage == 1) {
    if (tile == 9) fill_tma<SOLVER, 1, 32, 6, 3, 4>(out);
    else fill_tma<SOLVER, 1, 32, 8, 3, 3>(out);
    return true;
  }
  return pick_variant<3, float, 32, 7, 4>(SOLVER, stage, out);
}

}  // namespace

bool stage_variant_3d_f32_tma(int solver, int stage, int tile, StageVariant* out) {
  if (tile != 9 && tile != 10) return false;
  if (solver == SOLVER_HLL) return pick_tma<SOLVER_HLL>(tile, stage, out);
  if (solver == SOLVER_HLLC) return pick_tma<SOLVER_HLLC>(tile, stage, out);
  return false;
}

}  // namespace gh
