// Shared-memory-tiled FP32 stencil rows (tile.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace hhg {

// sets the shared-memory size attribute of every tiled kernel; call once
// before the first launch, outside stream capture
void tile_init();

// FP32 rows of op (OP_FULL in MODE_SET / MODE_RES, OP_BT / OP_BC in MODE_RES)
// by the tiled kernels, one launch per block type of the operator; `tab` is
// the level's FastTab<float, N> image of op.  Returns false (nothing launched)
// for other combinations.
bool tile_rows(int disc, int varnu, int op, int mode, const Geo& g, const OpDev& od, const void* tab, const float* x,
               const float* b, float* y, double alpha, cudaStream_t s);

}  // namespace hhg
