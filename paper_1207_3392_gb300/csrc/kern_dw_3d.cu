// kern_dw_3d.cu -- 3D stage kernels with the double-word (FP32 pair)
// arithmetic of dword.cuh.  Every value takes two registers: tiles 0 and 3
// cap the allocation at 128 registers (two 256-thread or four 128-thread CTAs
// per SM), tiles 1 and 2 leave it loose.
#include "instantiate.cuh"

namespace gh {

bool stage_variant_dw_3d(int solver, int stage, int tile, StageVariant* out) {
  switch (tile) {
    case 0: return pick_variant<3, dw, 32, 8, 2>(solver, stage, out);
    case 1: return pick_variant<3, dw, 32, 4, 2>(solver, stage, out);
    case 2: return pick_variant<3, dw, 32, 8, 1>(solver, stage, out);
    case 3: return pick_variant<3, dw, 32, 4, 4>(solver, stage, out);
  }
  return false;
}

}  // namespace gh
