// Cluster-resident inexact Uzawa smoother for small levels (small.cu).
#pragma once

#include <cuda_runtime.h>

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

// `iterations` inexact Uzawa iterations of a level in one cluster launch;
// returns 0 or -1 (launch failure).  Levels with more than 5^3 sites use the
// per-phase kernels instead.
template <class T>
int uzawa_cluster(int disc, int varnu, const Geo& g, T* x, const T* b, T* tmp, const double* inv_ml,
                  const SmallArgs& a, const OpDev& bc_op, const void* tabs, cudaStream_t s);

constexpr int64_t kSmallLevelSites = 5 * 5 * 5;

}  // namespace hhg
