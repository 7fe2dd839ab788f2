// Specialised stencil kernels (fast.cu): compile-time row structure,
// weights and linear offsets passed as __grid_constant__ parameters.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace hhg {

// weights and linear offsets (array * array_stride + di + dj sx + dk sy) of
// the interior terms of one operator on one level, in table order
template <class T, int N>
struct FastTab {
  T w[N];
  int off[N];
};

// launch shape of the specialised kernels on one level (autotuned)
struct Shape {
  int row_threads = 128;   // threads per block of the row kernels (64 / 128 / 256)
  int row_kplanes = 2;     // k planes per thread of the row kernels
  int gs_threads = 128;    // threads per block of the Gauss-Seidel kernels
  int gs_lanes = 1;        // lanes sharing the terms of one Gauss-Seidel site (1, 2, 4): edge groups
  int gs_lanes0 = 1;       // the same for the vertex group (its colour phases)
  int gs_threads0 = 0;     // threads per block of the vertex colour phases (0 = gs_threads)
  // own row shapes (threads, k planes, sites per thread) of the B^T and the
  // (B, -C) rows in the V-cycle precision; 0 = the full operator's
  int bt_threads = 0, bt_kplanes = 0, bt_sites = 0;
  int bc_threads = 0, bc_kplanes = 0, bc_sites = 0;
  // streaming kernels (stream.cu) of the FULL, B^T and (B, -C) rows: threads
  // per block (0 = the plain kernels), in the V-cycle precision (st_threads)
  // and in FP64 (st64_threads; the mixed solve's outer residual)
  int st_threads[3] = {0, 0, 0};
  int st64_threads[3] = {0, 0, 0};
  int st_sites[3] = {4, 4, 4};   // sites per thread of the FP32 streaming kernels (2 or 4)
  int row_sites = 1;       // sites per thread of the FP32 row kernels (1, or 4: four runs of 32 positions per warp)
  int row_sites64 = 1;     // the same for the FP64 row kernels
  // order of the per-phase Gauss-Seidel launches of a smoothing step: 0 = every
  // phase on the three components at once; 1 = component by component (all
  // sweeps of one component before the next: its arrays stay in L2 on levels
  // whose vectors exceed it)
  int gs_comp_major = 0;
};

// number of interior terms of a specialised operator (-1 if none)
int fast_terms(int disc, int varnu, int op);

// rows of OP_FULL / OP_BT / OP_BC (mode: MODE_SET / MODE_RES / MODE_ADD);
// `tab` points to a host FastTab<T, fast_terms(...)>
template <class T>
void fast_rows(int disc, int varnu, int op, const Geo& g, const OpDev& od, const void* tab, int mode, const T* x,
               const T* b, T* y, double alpha, const Shape& sh, cudaStream_t s);

// one Gauss-Seidel phase (group, colour) on the three velocity components
// (comp = -1) or on velocity component comp (0..2) only (A is block diagonal
// over the components, so each component's iterates are the same either
// way); `tab` points to a host FastTab<T, fast_terms(disc, varnu, OP_A)>
template <class T>
void fast_gs(int disc, int varnu, const Geo& g, const void* tab, int grp, int colour, double inv_diag, T* u,
             const T* rhs, const Shape& sh, cudaStream_t s, int comp = -1);

// the same two calls as work items of a batch being recorded (batch.h): the
// batched kernels live in their own translation units
template <class T>
void fast_rows_record(int disc, int varnu, int op, const Geo& g, const OpDev& od, const void* tab, int mode,
                      const T* x, const T* b, T* y, double alpha, const Shape& sh);
template <class T>
void fast_gs_record(int disc, int varnu, const Geo& g, const void* tab, int grp, int colour, double inv_diag, T* u,
                    const T* rhs, const Shape& sh, int comp);

}  // namespace hhg
