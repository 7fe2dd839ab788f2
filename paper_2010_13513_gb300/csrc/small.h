// Shared-memory-resident inexact Uzawa smoother for small levels (small.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace hhg {

// scalar arguments of one smoother launch
struct SmallArgs {
  int iterations;          // Uzawa iterations
  int xi;                  // Gauss-Seidel sweeps per velocity step
  int ahat;                // HHG_AHAT_F / HHG_AHAT_S
  double inv_omega_inv;    // omega = 1 / omega^{-1}
  double inv_diag[8];      // 1 / diag(A) per group
};

// one stencil row of the smoother's operators: output array, output group,
// whether boundary sites are computed (else set to 0), its interior terms
// [t0, t0 + n0 + n1 + n2) in three segments (unscaled, x e^{+}, x e^{-}), and
// its per-cube boundary terms [bs, bs + bn) of segment 2 in the op's bterms
struct ResRow {
  int out, og, all, t0, n0, n1, n2, bs, bn;
};

constexpr int kResMaxTerms = 640;
constexpr int kResMaxRows = 24;

// parameter block of one launch: the component-0 rows of A per velocity
// group (all terms in segment 1, the diagonal first), the 3G rows of B^T,
// the pressure row of (B, -C), and their terms with offsets in the slab's
// local array stride (array * arr_l + di + dj sx + dk sy)
template <class T>
struct ResTabs {
  int G, nbt, nw, varnu;
  ResRow A[8];
  ResRow BT[kResMaxRows];
  ResRow BC;
  T w[kResMaxTerms];
  int off[kResMaxTerms];
};

constexpr int kResidentThreads = 1024;            // most threads per CTA (128..1024, a multiple of 32)
constexpr int kResidentMaxCtas = 16;              // largest (non-portable) cluster
constexpr size_t kResidentSmemMax = 225 * 1024;   // dynamic shared memory per CTA (static use below 2 KB)

// Slab decomposition: CTA c of a cluster of C owns the k planes
// [c (nz+1) / C, (c+1) (nz+1) / C) of every array of the block vector and
// keeps them, with one halo plane below and above, in shared memory, next to
// the residuals and omega M_L^{-1} of its owned planes.  Local array strides
// (elements) of the slab and of the owned-plane arrays, and shared memory per
// CTA (bytes, including the tables):
int64_t resident_arr(const Geo& g, int ctas);
int64_t resident_arr_t(const Geo& g, int ctas);
size_t resident_smem(const Geo& g, int ctas, int prec);
// true if `ctas` CTAs can hold the level (every CTA owns a plane, the slab
// fits the shared memory, the cluster can be scheduled).  Sets the kernel's
// shared-memory and cluster-size attributes; call before any launch with
// this CTA count and outside stream capture.
bool resident_feasible(int prec, const Geo& g, int ctas);

// `iterations` inexact Uzawa iterations of a level in one launch of a
// cluster of `ctas` CTAs of `threads` threads; `tabs` built for
// resident_arr(g, ctas).  Returns 0 or -1 (launch failure).
template <class T>
int uzawa_resident(const Geo& g, int ctas, int threads, T* x, const T* b, const double* inv_ml, const SmallArgs& a,
                   const OpDev& bc_op, const ResTabs<T>& tabs, cudaStream_t s);

}  // namespace hhg
