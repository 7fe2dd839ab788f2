// Refinement residual of the mixed-precision solve in double-float
// arithmetic (dfres.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

namespace hhg {

// whether the double-float residual covers this operator (the full operator
// of P1-P1 or P2-P1, constant or variable viscosity)
bool df_supported(int disc, int varnu);

// the kernel's parameter block (weights split into two FP32 numbers, linear
// offsets) from the FP64 specialised-kernel table of the full operator (a
// FastTab<double, N> image); false if the operator is not covered
bool df_table(int disc, int varnu, const std::vector<char>& ftab64, std::vector<char>& out);

// r = fl32(b - calA x) for the full operator of one level, with calA x
// accumulated in double-float arithmetic; xh, xl: scratch of n = (3G + 1) arr
// floats each (they receive the two FP32 parts of x).  od: the level's
// generic tables (per-cube terms of the boundary pressure rows).  While a
// batch records, the two kernels are recorded as work items (batched
// variants kb_split_df, kb_res_df) that merge with other problems' ones.
void df_residual(int disc, int varnu, const Geo& g, const OpDev& od, const std::vector<char>& dftab, const double* x,
                 const double* b, float* xh, float* xl, float* r, cudaStream_t s);

}  // namespace hhg
