// batch_registry.h -- compiled variants of the persistent batch kernel.
#pragma once

#include <stddef.h>

namespace gh {

struct BatchVariant {
  const void* fn;
  size_t smem;
  int tx;    // threads per CTA (one tile row)
  int cols;  // columns of cells a tile owns (tx - 1)
};

int batch_tile_count();
bool batch_variant_f32(int solver, int stage, int tile, BatchVariant* out);
bool batch_variant_f64(int solver, int stage, int tile, BatchVariant* out);
bool batch_variant_dw(int solver, int stage, int tile, BatchVariant* out);

}  // namespace gh
