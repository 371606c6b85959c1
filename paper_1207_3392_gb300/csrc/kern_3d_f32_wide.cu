// kern_3d_f32_wide.cu -- 3D FP32 stage kernels on 512-thread tiles (less halo
// per cell; one CTA per SM may use up to 128 registers a thread).
#include "instantiate.cuh"

namespace gh {

bool stage_variant_3d_f32_wide(int solver, int stage, int tile, StageVariant* out) {
  switch (tile) {
    case 4: return pick_variant<3, float, 32, 16, 1>(solver, stage, out);
    case 5: return pick_variant<3, float, 64, 8, 1>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
