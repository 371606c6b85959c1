// kern_3d_f32.cu -- 3D stage kernels, FP32 storage with FP64 recovery.
#include "instantiate.cuh"

namespace gh {

int tile_count_3d() { return 3; }

bool stage_variant_3d_f32(int solver, int stage, int tile, StageVariant* out) {
  switch (tile) {
    case 0: return pick_variant<3, float, 32, 8>(solver, stage, out);
    case 1: return pick_variant<3, float, 32, 4>(solver, stage, out);
    case 2: return pick_variant<3, float, 64, 4>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
