// Launch wrappers of the HHG Stokes kernels (implemented in kernels.cu).
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace hhg {

enum ApplyMode { MODE_SET = 0, MODE_RES = 1, MODE_ADD = 2 };
enum ReduceMode { RED_SQ = 0, RED_DOT = 1, RED_WSUM = 2, RED_SUM = 3 };

// stencil rows: y (=, b -, += alpha) Op x over all rows of `op`
template <class T>
void launch_apply(const Geo& g, const OpDev& op, int mode, const T* x, const T* b, T* y, double alpha,
                  cudaStream_t s);

// the same on the rows within one site of the box's faces only: exact when x
// is non-zero only on boundary nodes (the Dirichlet lifting), since the rows
// farther inside read no boundary node
template <class T>
void launch_apply_shell(const Geo& g, const OpDev& op, int mode, const T* x, const T* b, T* y, double alpha,
                        cudaStream_t s);

// one multicolour Gauss-Seidel phase on the three velocity components:
// group `grp`, colour `colour` (0..3 for the vertex group, -1 = whole group)
template <class T>
void launch_gs(const Geo& g, const OpDev& A, int grp, int colour, double inv_diag, T* u, const T* rhs,
               cudaStream_t s);

// p -= r * inv_mlhat / omega_inv on all pressure nodes
template <class T>
void launch_pupdate(const Geo& g, T* p, const T* r, const double* inv_mlhat, double inv_omega_inv, cudaStream_t s);

// xf[base_f..] += I xc (interior_only: Dirichlet DoFs of xf untouched)
template <class T>
void launch_prolong(const Geo& gf, const Geo& gc, const XferDev& X, int base_f, int base_c, int ncomp, int G,
                    bool interior_only, const T* xc, T* xf, cudaStream_t s);

// rc[base_c..] = I^T rf (interior_only: Dirichlet rows set to 0)
// canonical host order (3 velocity components over the velocity nodes, then
// the pressure nodes) <-> padded layout; the scatter writes only the nodes
// (only boundary velocity nodes if boundary_only), the target is pre-zeroed
template <class T>
void launch_canon_scatter(const Geo& g, const double* src, T* dst, int64_t nvn, int64_t npn, bool with_pressure,
                          bool boundary_only, cudaStream_t s);
template <class T>
void launch_canon_gather(const Geo& g, const T* src, double* dst, int64_t nvn, int64_t npn, cudaStream_t s);
template <class T>
void launch_restrict(const Geo& gf, const Geo& gc, const XferDev& X, int base_f, int base_c, int ncomp, int G,
                     bool interior_only, const T* rf, T* rc, cudaStream_t s);

// deterministic two-pass reduction over n contiguous elements into out[0]
template <class T>
void launch_reduce(int mode, const T* a, const T* b, const double* w, int64_t n, double* partials, int max_blocks,
                   double* out, cudaStream_t s);

// p -= (*sum) * scale on all pressure nodes
template <class T>
void launch_sub_scalar_p(const Geo& g, T* p, const double* sum, double scale, cudaStream_t s);

// x[idx[r]] = sum_j Z[r, j] b[idx[j]]
template <class T>
void launch_coarse(const double* Z, int n, const int64_t* idx, const T* b, T* x, cudaStream_t s);

// element-wise helpers over n contiguous elements
void launch_cast_d2f(const double* a, float* b, int64_t n, cudaStream_t s);
void launch_add_f2d(const float* a, double* b, int64_t n, cudaStream_t s);
template <class T>
void launch_axpy(double alpha, const T* x, T* y, int64_t n, cudaStream_t s);   // y += alpha x
template <class T>
void launch_xpby(const T* x, double beta, const T* y, T* z, int64_t n, cudaStream_t s);  // z = x + beta y
void launch_inv(const double* a, double* b, int64_t n, cudaStream_t s);        // b = 1/a where a != 0
// bytes (a multiple of 4) of zeros at p (cudaMemsetAsync; a merged op while a batch records)
cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s);

extern thread_local int64_t g_launches;   // kernels issued by this thread

}  // namespace hhg
