// kern_dw.cu -- 1D and 2D stage kernels with the double-word (FP32 pair)
// arithmetic of dword.cuh.
#include "instantiate.cuh"

namespace gh {

int tile_count_dw(int ndim) { return ndim == 3 ? 4 : 1; }

bool stage_variant_dw(int ndim, int solver, int stage, int tile, StageVariant* out) {
  if (ndim == 3) return stage_variant_dw_3d(solver, stage, tile, out);
  if (tile != 0) return false;
  return ndim == 1 ? pick_variant<1, dw, 128, 1>(solver, stage, out) : pick_variant<2, dw, 128, 1>(solver, stage, out);
}

}  // namespace gh
