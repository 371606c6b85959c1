// kern_1d.cu -- 1D stage-kernel instantiations (tiles of TX cells).
#include "instantiate.cuh"

namespace gh {

int tile_count_1d() { return 2; }

bool stage_variant_1d(bool fp64, int solver, int stage, int tile, StageVariant* out) {
  switch (tile) {
    case 0: return fp64 ? pick_variant<1, double, 128, 1>(solver, stage, out)
                        : pick_variant<1, float, 128, 1>(solver, stage, out);
    case 1: return fp64 ? pick_variant<1, double, 256, 1>(solver, stage, out)
                        : pick_variant<1, float, 256, 1>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
