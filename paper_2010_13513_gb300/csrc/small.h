// Shared-memory-resident inexact Uzawa smoother for small levels (small.cu).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "fast.h"
#include "internal.h"
#include "structure.inc"

namespace hhg {

// scalar arguments of one smoother launch
struct SmallArgs {
  int iterations;          // Uzawa iterations
  int xi;                  // Gauss-Seidel sweeps per velocity step
  int ahat;                // HHG_AHAT_F / HHG_AHAT_S
  double inv_omega_inv;    // omega = 1 / omega^{-1}
  double inv_diag[8];      // 1 / diag(A) per group
};

// the parameter tables of the three operators used by the smoother
template <int DISC, int VARNU, class T>
struct SmallTabs {
  FastTab<T, gen::S<DISC, VARNU, OP_A>::N> A;
  FastTab<T, gen::S<DISC, VARNU, OP_BT>::N> BT;
  FastTab<T, gen::S<DISC, VARNU, OP_BC>::N> BC;
};

size_t small_tabs_bytes(int disc, int varnu, int prec);
size_t small_tabs_offset(int disc, int varnu, int prec, int which);   // 0 = A, 1 = BT, 2 = BC

constexpr int kResidentThreads = 1024;            // threads per CTA
constexpr int kResidentMaxCtas = 16;              // largest (non-portable) cluster
constexpr size_t kResidentSmemMax = 227 * 1024;   // dynamic shared memory per CTA

// Slab decomposition: CTA c of a cluster of C owns the k planes
// [c (nz+1) / C, (c+1) (nz+1) / C) of every array of the block vector and
// keeps them, with one halo plane below and above, in shared memory.  Local
// array stride (elements) and shared memory per CTA (bytes):
int64_t resident_arr(const Geo& g, int ctas);
size_t resident_smem(const Geo& g, int ctas, int prec);
// true if `ctas` CTAs can hold the level (every CTA owns a plane, the slab
// fits the shared memory, the cluster can be scheduled).  Sets the kernel's
// shared-memory and cluster-size attributes; call before any launch with
// this CTA count and outside stream capture.
bool resident_feasible(int disc, int varnu, int prec, const Geo& g, int ctas);
// rewrites the linear offsets (array * arr_g + rel) of a SmallTabs image to
// the local array stride arr_l; false if a term reaches beyond the adjacent
// sites (then the slab layout would not hold it)
bool small_tabs_localise(int disc, int varnu, int prec, const std::vector<char>& in, const Geo& g, int64_t arr_l,
                         std::vector<char>& out);

// `iterations` inexact Uzawa iterations of a level in one launch of a
// cluster of `ctas` CTAs; `tabs` is a SmallTabs image localised to
// resident_arr(g, ctas).  Returns 0 or -1 (launch failure).
template <class T>
int uzawa_resident(int disc, int varnu, const Geo& g, int ctas, T* x, const T* b, T* tmp, const double* inv_ml,
                   const SmallArgs& a, const OpDev& bc_op, const void* tabs, cudaStream_t s);

}  // namespace hhg
