// kern_2d.cu -- 2D stage-kernel instantiations (row tiles of TX cells that march along y).
#include "instantiate.cuh"

namespace gh {

int tile_count_2d() { return 3; }

bool stage_variant_2d(bool fp64, int solver, int stage, int tile, StageVariant* out) {
  if (solver == SOLVER_HLLC_SW)
    return tile == 0 && (fp64 ? pick_switch<2, double, 128, 1>(stage, out) : pick_switch<2, float, 128, 1>(stage, out));
  switch (tile) {
    case 0: return fp64 ? pick_variant<2, double, 128, 1>(solver, stage, out)
                        : pick_variant<2, float, 128, 1>(solver, stage, out);
    case 1: return fp64 ? pick_variant<2, double, 64, 1>(solver, stage, out)
                        : pick_variant<2, float, 64, 1>(solver, stage, out);
    case 2: return fp64 ? pick_variant<2, double, 256, 1>(solver, stage, out)
                        : pick_variant<2, float, 256, 1>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
