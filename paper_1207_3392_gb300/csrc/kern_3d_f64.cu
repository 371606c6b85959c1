// kern_3d_f64.cu -- 3D stage kernels, FP64 throughout.
#include "instantiate.cuh"

namespace gh {

int tile_count_3d_f64() { return 4; }

bool stage_variant_3d_f64(int solver, int stage, int tile, StageVariant* out) {
  if (solver == SOLVER_HLLC_SW) return tile == 0 && pick_switch<3, double, 32, 8>(stage, out);
  switch (tile) {
    case 0: return pick_variant<3, double, 32, 8>(solver, stage, out);
    case 1: return pick_variant<3, double, 32, 4>(solver, stage, out);
    case 2: return pick_variant<3, double, 64, 4>(solver, stage, out);
    case 3: return pick_variant<3, double, 32, 4, 2>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
