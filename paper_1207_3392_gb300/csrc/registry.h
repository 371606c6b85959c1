// registry.h -- host-side table of the compiled stage-kernel variants.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace gh {

// One compiled instantiation of hydro_stage_kernel.
struct StageVariant {
  const void* fn;      // kernel entry
  size_t smem;         // dynamic shared memory per CTA (bytes)
  int tx, ty;          // tile shape in cells
  int threads;         // threads per CTA
  int tma = 0;         // 1: takes TmaStageArgs (state planes staged by TMA), see stage_tma.cuh
  int box_x = 0, box_y = 0;  // TMA box of one plane (cells along x and y)
  int pair = 0;        // 1: two march planes per thread (stage_pair.cuh); chunks of an even plane count
};

// Tile shapes compiled per dimensionality and precision (GENASIS_FP64,
// GENASIS_FP32_MIXED, GENASIS_FP64_DW); index `tile` selects one.
int stage_tile_count(int ndim, int prec);
// Fills *out for (ndim, precision, solver, stage, tile); returns false if absent.
bool stage_variant(int ndim, int prec, int solver, int stage, int tile, StageVariant* out);
bool stage_variant_dw(int ndim, int solver, int stage, int tile, StageVariant* out);
bool stage_variant_dw_3d(int solver, int stage, int tile, StageVariant* out);
int tile_count_dw(int ndim);

bool stage_variant_1d(bool fp64, int solver, int stage, int tile, StageVariant* out);
bool stage_variant_2d(bool fp64, int solver, int stage, int tile, StageVariant* out);
bool stage_variant_3d_f32(int solver, int stage, int tile, StageVariant* out);
bool stage_variant_3d_f32_wide(int solver, int stage, int tile, StageVariant* out);
bool stage_variant_3d_f32_tma(int solver, int stage, int tile, StageVariant* out);
bool stage_variant_3d_f32_pair(int solver, int stage, int tile, StageVariant* out);
bool stage_variant_3d_f64(int solver, int stage, int tile, StageVariant* out);
int tile_count_1d();
// One-launch advance of small 1D meshes (kern_1d_advance.cu): the
// kernel for (precision, solver) on tx threads and its dynamic shared memory,
// or nullptr if not compiled.
const void* advance_1d_kernel(bool fp64, int solver, int tx, size_t* smem);
int tile_count_2d();
int tile_count_3d_f32();
int tile_count_3d_f64();

}  // namespace gh
