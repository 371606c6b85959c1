// kern_3d_f32.cu -- 3D stage kernels, FP32 storage with FP64 recovery.
#include "instantiate.cuh"

namespace gh {

int tile_count_3d_f32() { return 14; }

// Register caps: 256-thread tiles at 3 CTAs per SM and 128-thread tiles at 6
// (80 registers, 24 resident warps); tile 3 keeps the uncapped allocation;
// tile 7 caps at 64 registers (32 warps, some spills); tile 8, 32 x 7 at 4
// CTAs per SM, holds 72 registers without spilling (28 warps) and is the
// fastest at 256^3; tile 6 forms the in-plane slopes per face (no face-state
// phase); tiles 4 and 5 (512 threads) are in kern_3d_f32_wide.cu, tiles 9
// and 10 (the state planes staged by TMA) in kern_3d_f32_tma.cu, tiles 11 to
// 13 (two march planes per thread, packed FP32) in kern_3d_f32_pair.cu.  16 x 16,
// 32 x 12, 32 x 14, 32 x 13 and 32 x 9 tiles were measured and lost.
bool stage_variant_3d_f32(int solver, int stage, int tile, StageVariant* out) {
  if (solver == SOLVER_HLLC_SW) {
    if (tile == 0) return pick_switch<3, float, 32, 8, 3>(stage, out);
    if (tile == 8) return pick_switch<3, float, 32, 7, 4>(stage, out);
    return false;
  }
  switch (tile) {
    case 0: return pick_variant<3, float, 32, 8, 3>(solver, stage, out);
    case 1: return pick_variant<3, float, 32, 4, 6>(solver, stage, out);
    case 2: return pick_variant<3, float, 64, 4, 3>(solver, stage, out);
    case 3: return pick_variant<3, float, 32, 8, 2>(solver, stage, out);
    case 6: return pick_variant<3, float, 32, 8, 3, false>(solver, stage, out);
    case 7: return pick_variant<3, float, 32, 8, 4>(solver, stage, out);
    case 8: return pick_variant<3, float, 32, 7, 4>(solver, stage, out);
  }
  if (tile == 9 || tile == 10) return stage_variant_3d_f32_tma(solver, stage, tile, out);
  if (tile >= 11 && tile <= 13) return stage_variant_3d_f32_pair(solver, stage, tile, out);
  return stage_variant_3d_f32_wide(solver, stage, tile, out);
}

}  // namespace gh
