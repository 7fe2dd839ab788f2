// CUDA kernels of the HHG Stokes library (sm_103a).
//
// All kernels work on the box-shaped group arrays described in internal.h.
// One thread owns one DoF site (coarse index (i,j,k)); consecutive threads
// of a warp own consecutive i, so every stencil term is one coalesced load
// of 32 consecutive elements.  Stencil tables are warp-uniform reads of a few
// KB that stay in L1.  Reductions are deterministic (fixed grid, fixed
// order of the final pass).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "batch.h"
#include "kernels.h"

namespace hhg {

thread_local int64_t g_launches = 0;

namespace {

template <class T> __device__ __forceinline__ T wsel(const double* w64, const float* w32, int t);
template <> __device__ __forceinline__ double wsel<double>(const double* w64, const float*, int t) { return __ldg(w64 + t); }
template <> __device__ __forceinline__ float wsel<float>(const double*, const float* w32, int t) { return __ldg(w32 + t); }

__device__ __forceinline__ int64_t site_index(const Geo& g, int i, int j, int k) {
  return int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy;
}

// DoF at coarse index (i,j,k) of group offset (ox,oy,oz): valid and on the boundary?
__device__ __forceinline__ bool dof_valid(const Geo& g, int i, int j, int k, int ox, int oy, int oz) {
  return i <= g.nx - ox && j <= g.ny - oy && k <= g.nz - oz && i >= 0 && j >= 0 && k >= 0;
}
__device__ __forceinline__ bool dof_boundary(const Geo& g, int i, int j, int k, int ox, int oy, int oz) {
  const int Px = 2 * i + ox, Py = 2 * j + oy, Pz = 2 * k + oz;
  return Px == 0 || Py == 0 || Pz == 0 || Px == 2 * g.nx || Py == 2 * g.ny || Pz == 2 * g.nz;
}

__constant__ int c_goff[8][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

// ------------------------------------------------------------------ apply
// row r of op at coarse index (i, j, k)
template <class T, int MODE>
__device__ __forceinline__ void apply_site(const Geo& g, const OpDev& op, int r, int i, int j, int k,
                                           const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y,
                                           T alpha) {
  const DRow row = op.rows[r];
  const int ox = c_goff[row.og][0], oy = c_goff[row.og][1], oz = c_goff[row.og][2];
  if (!dof_valid(g, i, j, k, ox, oy, oz)) return;
  const int64_t idx = site_index(g, i, j, k);
  T* yo = y + int64_t(row.out_arr) * g.arr + idx;
  const bool bnd = dof_boundary(g, i, j, k, ox, oy, oz);
  T acc[3] = {T(0), T(0), T(0)};
  if (!bnd) {
    int t = row.t0;
    const int ns[3] = {row.n0, row.n1, row.n2};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      T a = T(0);
      for (int e = 0; e < ns[s]; ++e, ++t) {
        const DTerm tm = op.terms[t];
        a += wsel<T>(op.w64, op.w32, t) * x[int64_t(tm.arr) * g.arr + idx + tm.off];
      }
      acc[s] = a;
    }
  } else if (row.all_rows) {
    int t = row.b0;
    const int ms[3] = {row.m0, row.m1, row.m2};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      T a = T(0);
      for (int e = 0; e < ms[s]; ++e, ++t) {
        const DTermB tm = op.bterms[t];
        const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
        if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
        a += wsel<T>(op.bw64, op.bw32, t) * x[int64_t(tm.arr) * g.arr + idx + tm.off];
      }
      acc[s] = a;
    }
  } else {
    if (MODE != MODE_ADD) *yo = T(0);
    return;
  }
  T v = acc[0];
  if (g.nu_ah != 0.0) {
    v += T(g.esc[k]) * acc[1] + T(g.eisc[k]) * acc[2];
  } else {
    v += acc[1] + acc[2];
  }
  if (MODE == MODE_SET) *yo = v;
  else if (MODE == MODE_RES) *yo = b[int64_t(row.out_arr) * g.arr + idx] - v;
  else *yo += alpha * v;
}

template <class T, int MODE>
__global__ void __launch_bounds__(128) k_apply(Geo g, OpDev op, const T* __restrict__ x, const T* __restrict__ b,
                                               T* __restrict__ y, T alpha) {
  const int nzp = g.nz + 1;
  const int r = blockIdx.z / nzp;
  const int k = blockIdx.z - r * nzp;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  apply_site<T, MODE>(g, op, r, i, j, k, x, b, y, alpha);
}

// the rows within one site of the box's faces (the shell, where an input that
// is non-zero only on boundary nodes gives non-zero rows): blockIdx.y = row x
// plane (planes k of `ks`: the first two and last two planes, all of each;
// or the inner planes, their ring of sites with i or j within one site of a
// face)
template <class T, int MODE>
__global__ void __launch_bounds__(128) k_apply_shell(Geo g, OpDev op, int inner, const T* __restrict__ x,
                                                     const T* __restrict__ b, T* __restrict__ y, T alpha) {
  const int np = inner ? g.nz - 3 : 4;
  const int r = blockIdx.y / np, kk = blockIdx.y - r * np;
  const int k = inner ? 2 + kk : (kk < 2 ? kk : g.nz - 3 + kk);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  const int nxp = g.nx + 1;
  int i, j;
  if (!inner) {
    if (q >= nxp * (g.ny + 1)) return;
    j = q / nxp;
    i = q - j * nxp;
  } else {
    const int nfull = 4 * nxp;                       // rows j = 0, 1, ny - 1, ny
    if (q < nfull) {
      const int jj = q / nxp;
      i = q - jj * nxp;
      j = jj < 2 ? jj : g.ny - 3 + jj;
    } else {
      const int q2 = q - nfull;                     // rows 2 .. ny - 2: i = 0, 1, nx - 1, nx
      j = 2 + q2 / 4;
      if (j > g.ny - 2) return;
      const int c = q2 - (j - 2) * 4;
      i = c < 2 ? c : g.nx - 3 + c;
    }
  }
  apply_site<T, MODE>(g, op, r, i, j, k, x, b, y, alpha);
}

// ------------------------------------------------------- Gauss-Seidel phase
template <class T>
__global__ void __launch_bounds__(128) k_gs(Geo g, OpDev A, int grp, int colour, T inv_diag, T* __restrict__ u,
                                            const T* __restrict__ rhs) {
  const int k = blockIdx.z;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int ox = c_goff[grp][0], oy = c_goff[grp][1], oz = c_goff[grp][2];
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (colour >= 0) i = 4 * i + (((colour - j - k) % 4) + 4) % 4;
  if (!dof_valid(g, i, j, k, ox, oy, oz) || dof_boundary(g, i, j, k, ox, oy, oz)) return;
  const int64_t idx = site_index(g, i, j, k);
  const DRow row = A.rows[grp];          // component-0 row of group grp; comps 1,2 shift by G arrays
  const int64_t cstride = int64_t(g.G) * g.arr;
  T a0 = T(0), a1 = T(0), a2 = T(0);
  for (int t = row.t0 + 1; t < row.t0 + row.n1; ++t) {     // all A terms are in seg 1, diagonal first
    const DTerm tm = A.terms[t];
    const T w = wsel<T>(A.w64, A.w32, t);
    const T* p = u + int64_t(tm.arr) * g.arr + idx + tm.off;
    a0 += w * p[0];
    a1 += w * p[cstride];
    a2 += w * p[2 * cstride];
  }
  T einv = T(1);
  if (g.nu_ah != 0.0) einv = T(g.eisc[k]);
  const int64_t o0 = int64_t(grp) * g.arr + idx;
  u[o0] = (rhs[o0] * einv - a0) * inv_diag;
  u[o0 + cstride] = (rhs[o0 + cstride] * einv - a1) * inv_diag;
  u[o0 + 2 * cstride] = (rhs[o0 + 2 * cstride] * einv - a2) * inv_diag;
}

// --------------------------------------------------------- pressure update
// Every kernel below is a device body that takes its block index (and grid
// size) as arguments, a plain kernel that passes blockIdx, and a batched
// kernel (kb_*) that runs the body for one work item of a merged launch.
template <class T>
struct PUpdateA { Geo g; T* p; const T* r; const double* inv_ml; double s; };
template <class T>
__device__ __forceinline__ void pupdate_body(const uint3 bid, const Geo& g, T* __restrict__ p, const T* __restrict__ r,
                                             const double* __restrict__ inv_ml, double s) {
  const int i = bid.x * blockDim.x + threadIdx.x;
  const int j = bid.y * blockDim.y + threadIdx.y;
  const int k = bid.z;
  if (i > g.nx || j > g.ny) return;
  const int64_t idx = site_index(g, i, j, k);
  p[idx] -= T(s * inv_ml[idx]) * r[idx];
}
template <class T>
__global__ void k_pupdate(Geo g, T* __restrict__ p, const T* __restrict__ r, const double* __restrict__ inv_ml,
                          double s) {
  pupdate_body<T>(blockIdx, g, p, r, inv_ml, s);
}
template <class T>
__global__ void kb_pupdate(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<PUpdateA<T>>(items, n, bid, gd);
  pupdate_body<T>(bid, it.a.g, it.a.p, it.a.r, it.a.inv_ml, it.a.s);
}

template <class T>
struct SubScalarA { Geo g; T* p; const double* sum; double scale; };
template <class T>
__device__ __forceinline__ void sub_scalar_body(const uint3 bid, const Geo& g, T* __restrict__ p,
                                                const double* __restrict__ sum, double scale) {
  const int i = bid.x * blockDim.x + threadIdx.x;
  const int j = bid.y * blockDim.y + threadIdx.y;
  const int k = bid.z;
  if (i > g.nx || j > g.ny) return;
  p[site_index(g, i, j, k)] -= T(sum[0] * scale);
}
template <class T>
__global__ void k_sub_scalar_p(Geo g, T* __restrict__ p, const double* __restrict__ sum, double scale) {
  sub_scalar_body<T>(blockIdx, g, p, sum, scale);
}
template <class T>
__global__ void kb_sub_scalar_p(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<SubScalarA<T>>(items, n, bid, gd);
  sub_scalar_body<T>(bid, it.a.g, it.a.p, it.a.sum, it.a.scale);
}

// ---------------------------------------------------------------- transfers
template <class T>
struct XferA { Geo gf, gc; XferDev X; int base_f, base_c, ncomp, G, interior_only; const T* in; T* out; };
template <class T>
__device__ __forceinline__ void prolong_body(const uint3 bid, const Geo& gf, const Geo& gc, const XferDev& X,
                                             int base_f, int base_c, int ncomp, int G, int interior_only,
                                             const T* __restrict__ xc, T* __restrict__ xf) {
  const int nzp = gf.nz + 1;
  const int gfi = bid.z / nzp;
  const int k = bid.z - gfi * nzp;
  const int i = bid.x * blockDim.x + threadIdx.x;
  const int j = bid.y * blockDim.y + threadIdx.y;
  const int ox = G == 1 ? 0 : c_goff[gfi][0], oy = G == 1 ? 0 : c_goff[gfi][1], oz = G == 1 ? 0 : c_goff[gfi][2];
  if (!dof_valid(gf, i, j, k, ox, oy, oz)) return;
  if (interior_only && dof_boundary(gf, i, j, k, ox, oy, oz)) return;
  int ax, ay, az, cls;
  if (X.order == 2) {
    const int Px = 2 * i + ox, Py = 2 * j + oy, Pz = 2 * k + oz;
    ax = Px >> 2; ay = Py >> 2; az = Pz >> 2;
    cls = (Px & 3) + 4 * ((Py & 3) + 4 * (Pz & 3));
  } else {
    ax = i >> 1; ay = j >> 1; az = k >> 1;
    cls = (i & 1) + 2 * ((j & 1) + 2 * (k & 1));
  }
  const int64_t cidx = site_index(gc, ax, ay, az);
  const int64_t fidx = site_index(gf, i, j, k);
  const int t0 = X.pcls_start[cls], t1 = X.pcls_start[cls + 1];
  const int64_t cstride_c = int64_t(G) * gc.arr, cstride_f = int64_t(G) * gf.arr;
  for (int c = 0; c < ncomp; ++c) {
    T a = T(0);
    for (int t = t0; t < t1; ++t) {
      const DXTerm tm = X.pterms[t];
      const int64_t off = int64_t(tm.di) + int64_t(tm.dj) * gc.sx + int64_t(tm.dk) * gc.sy;
      a += wsel<T>(X.pw64, X.pw32, t) * xc[int64_t(base_c + tm.arr) * gc.arr + c * cstride_c + cidx + off];
    }
    xf[int64_t(base_f + gfi) * gf.arr + c * cstride_f + fidx] += a;
  }
}
template <class T>
__global__ void __launch_bounds__(128) k_prolong(Geo gf, Geo gc, XferDev X, int base_f, int base_c, int ncomp, int G,
                                                 int interior_only, const T* __restrict__ xc, T* __restrict__ xf) {
  prolong_body<T>(blockIdx, gf, gc, X, base_f, base_c, ncomp, G, interior_only, xc, xf);
}
template <class T>
__global__ void __launch_bounds__(128) kb_prolong(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<XferA<T>>(items, n, bid, gd);
  const XferA<T>& a = it.a;
  prolong_body<T>(bid, a.gf, a.gc, a.X, a.base_f, a.base_c, a.ncomp, a.G, a.interior_only, a.in, a.out);
}

// r_c = I^T r_f per coarse DoF: its restriction terms (up to 125 for the P2
// vertex group) are shared by P lanes, lane p taking terms p, p+P, ..., and
// the partial sums are added by shuffles.  Block: 128 threads = 128/P coarse
// sites along i; grid: (i blocks, j, (k, group)).
template <class T, int P>
__device__ __forceinline__ void restrict_body(const uint3 bid, const Geo& gf, const Geo& gc, const XferDev& X,
                                              int base_f, int base_c, int ncomp, int G, int interior_only,
                                              const T* __restrict__ rf, T* __restrict__ rc) {
  const int nzp = gc.nz + 1;
  const int gci = bid.z / nzp;
  const int k = bid.z - gci * nzp;
  const int i = bid.x * (128 / P) + int(threadIdx.x) / P, p = int(threadIdx.x) % P;
  const int j = bid.y;
  const int ox = G == 1 ? 0 : c_goff[gci][0], oy = G == 1 ? 0 : c_goff[gci][1], oz = G == 1 ? 0 : c_goff[gci][2];
  const bool valid = dof_valid(gc, i, j, k, ox, oy, oz);
  const bool zero = valid && interior_only && dof_boundary(gc, i, j, k, ox, oy, oz);
  const int64_t cstride_f = int64_t(G) * gf.arr;
  T a0 = T(0), a1 = T(0), a2 = T(0);
  if (valid && !zero) {
    const int t0 = X.rg_start[gci], t1 = X.rg_start[gci + 1];
#pragma unroll 4
    for (int t = t0 + p; t < t1; t += P) {
      const DXTerm tm = X.rterms[t];
      const int fi = 2 * i + tm.di, fj = 2 * j + tm.dj, fk = 2 * k + tm.dk;
      if (fi < -1 || fj < -1 || fk < -1 || fi > gf.nx + 1 || fj > gf.ny + 1 || fk > gf.nz + 1) continue;
      const T w = wsel<T>(X.rw64, X.rw32, t);
      const T* f = rf + int64_t(base_f + tm.arr) * gf.arr + site_index(gf, fi, fj, fk);
      a0 += w * f[0];
      if (ncomp > 1) {
        a1 += w * f[cstride_f];
        a2 += w * f[2 * cstride_f];
      }
    }
  }
#pragma unroll
  for (int m = P >> 1; m > 0; m >>= 1) {          // all lanes of the warp take part
    a0 += __shfl_xor_sync(0xffffffffu, a0, m);
    a1 += __shfl_xor_sync(0xffffffffu, a1, m);
    a2 += __shfl_xor_sync(0xffffffffu, a2, m);
  }
  if (!valid || p != 0) return;
  const int64_t cidx = site_index(gc, i, j, k), cstride_c = int64_t(G) * gc.arr;
  T* o = rc + int64_t(base_c + gci) * gc.arr + cidx;
  o[0] = zero ? T(0) : a0;
  if (ncomp > 1) {
    o[cstride_c] = zero ? T(0) : a1;
    o[2 * cstride_c] = zero ? T(0) : a2;
  }
}
template <class T, int P>
__global__ void __launch_bounds__(128) k_restrict(Geo gf, Geo gc, XferDev X, int base_f, int base_c, int ncomp, int G,
                                                  int interior_only, const T* __restrict__ rf, T* __restrict__ rc) {
  restrict_body<T, P>(blockIdx, gf, gc, X, base_f, base_c, ncomp, G, interior_only, rf, rc);
}
template <class T, int P>
__global__ void __launch_bounds__(128) kb_restrict(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<XferA<T>>(items, n, bid, gd);
  const XferA<T>& a = it.a;
  restrict_body<T, P>(bid, a.gf, a.gc, a.X, a.base_f, a.base_c, a.ncomp, a.G, a.interior_only, a.in, a.out);
}

// ------------------------------------------ canonical order <-> padded layout
// Canonical host order: 3 velocity components (component-major) over the
// velocity nodes in lexicographic order (P1: the lattice sites; P2: the
// doubled lattice, node (I,J,K) in group of parity (I&1, J&1, K&1) at site
// (I>>1, J>>1, K>>1)), then the pressure nodes (the lattice sites).
__constant__ int c_parity_group[8] = {0, 1, 2, 4, 3, 5, 6, 7};   // index ox | oy << 1 | oz << 2

struct CanonMap {
  int64_t off;      // element of the node in the layout vector
  bool bnd;         // on the domain boundary
};

// blockIdx.y: component 0..2 (velocity) or 3 (pressure); x: node index
__device__ __forceinline__ CanonMap canon_map(const Geo& g, int comp, int64_t ci) {
  CanonMap m;
  if (comp < 3 && g.G > 1) {
    const int64_t nI = 2 * int64_t(g.nx) + 1, nJ = 2 * int64_t(g.ny) + 1;
    const int64_t K = ci / (nI * nJ), rem = ci - K * nI * nJ, J = rem / nI, I = rem - J * nI;
    const int gg = c_parity_group[int(I & 1) | int(J & 1) << 1 | int(K & 1) << 2];
    m.off = int64_t(comp * g.G + gg) * g.arr + ((I >> 1) + 1) + ((J >> 1) + 1) * g.sx + ((K >> 1) + 1) * g.sy;
    m.bnd = I == 0 || J == 0 || K == 0 || I == 2 * g.nx || J == 2 * g.ny || K == 2 * g.nz;
  } else {
    const int64_t nI = g.nx + 1, nJ = g.ny + 1;
    const int64_t k = ci / (nI * nJ), rem = ci - k * nI * nJ, j = rem / nI, i = rem - j * nI;
    const int arr = comp < 3 ? comp * g.G : 3 * g.G;
    m.off = int64_t(arr) * g.arr + (i + 1) + (j + 1) * g.sx + (k + 1) * g.sy;
    m.bnd = i == 0 || j == 0 || k == 0 || i == g.nx || j == g.ny || k == g.nz;
  }
  return m;
}

template <class T>
__global__ void k_canon_scatter(Geo g, const double* __restrict__ src, T* __restrict__ dst, int64_t nvn, int64_t npn,
                                int boundary_only) {
  const int comp = blockIdx.y;
  const int64_t n = comp < 3 ? nvn : npn;
  for (int64_t ci = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; ci < n; ci += int64_t(gridDim.x) * blockDim.x) {
    const CanonMap m = canon_map(g, comp, ci);
    if (!boundary_only || m.bnd) dst[m.off] = T(src[comp * nvn + ci]);
  }
}

template <class T>
__global__ void k_canon_gather(Geo g, const T* __restrict__ src, double* __restrict__ dst, int64_t nvn, int64_t npn) {
  const int comp = blockIdx.y;
  const int64_t n = comp < 3 ? nvn : npn;
  for (int64_t ci = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; ci < n; ci += int64_t(gridDim.x) * blockDim.x)
    dst[comp * nvn + ci] = double(src[canon_map(g, comp, ci).off]);
}

// ---------------------------------------------------------------- reductions
template <class T>
struct ReduceA { const T* a; const T* b; const double* w; int64_t n; double* partials; };
template <class T, int MODE>
__device__ __forceinline__ void reduce_partial_body(const uint3 bid, const uint3 gd, const T* __restrict__ a,
                                                    const T* __restrict__ b, const double* __restrict__ w, int64_t n,
                                                    double* __restrict__ partials) {
  double s = 0.0;
  for (int64_t q = bid.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gd.x) * blockDim.x) {
    const double va = double(a[q]);
    if (MODE == RED_SQ) s += va * va;
    else if (MODE == RED_DOT) s += va * double(b[q]);
    else if (MODE == RED_WSUM) s += w[q] * va;
    else s += va;
  }
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) partials[bid.x] = s;
  }
}
template <class T, int MODE>
__global__ void __launch_bounds__(256) k_reduce_partial(const T* __restrict__ a, const T* __restrict__ b,
                                                        const double* __restrict__ w, int64_t n,
                                                        double* __restrict__ partials) {
  reduce_partial_body<T, MODE>(blockIdx, gridDim, a, b, w, n, partials);
}
template <class T, int MODE>
__global__ void __launch_bounds__(256) kb_reduce_partial(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<ReduceA<T>>(items, n, bid, gd);
  reduce_partial_body<T, MODE>(bid, gd, it.a.a, it.a.b, it.a.w, it.a.n, it.a.partials);
}

struct FinalA { const double* partials; int n; double* out; };
__device__ __forceinline__ void reduce_final_body(const double* __restrict__ partials, int n,
                                                  double* __restrict__ out) {
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += partials[q];
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[0] = s;
  }
}
__global__ void __launch_bounds__(256) k_reduce_final(const double* __restrict__ partials, int n,
                                                      double* __restrict__ out) {
  reduce_final_body(partials, n, out);
}
__global__ void __launch_bounds__(256) kb_reduce_final(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<FinalA>(items, n, bid, gd);
  reduce_final_body(it.a.partials, it.a.n, it.a.out);
}

// --------------------------------------------------------------- coarse solve
template <class T>
struct CoarseA { const double* Z; int n; const int64_t* idx; const T* b; T* x; };
template <class T>
__device__ __forceinline__ void coarse_body(const uint3 bid, const double* __restrict__ Z, int n,
                                            const int64_t* __restrict__ idx, const T* __restrict__ b,
                                            T* __restrict__ x) {
  const int r = bid.x;
  double s = 0.0;
  for (int q = threadIdx.x; q < n; q += blockDim.x) s += Z[int64_t(r) * n + q] * double(b[idx[q]]);
  __shared__ double sh[4];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) x[idx[r]] = T(sh[0] + sh[1] + sh[2] + sh[3]);
}
template <class T>
__global__ void __launch_bounds__(128) k_coarse(const double* __restrict__ Z, int n, const int64_t* __restrict__ idx,
                                                const T* __restrict__ b, T* __restrict__ x) {
  coarse_body<T>(blockIdx, Z, n, idx, b, x);
}
template <class T>
__global__ void __launch_bounds__(128) kb_coarse(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<CoarseA<T>>(items, n, bid, gd);
  coarse_body<T>(bid, it.a.Z, it.a.n, it.a.idx, it.a.b, it.a.x);
}

// ------------------------------------------------------------ element-wise
// grid-stride loops of the element-wise kernels: q runs over
// bid.x * blockDim.x + threadIdx.x, stepping by the item's grid
#define HHG_GRID_LOOP(q, n) \
  for (int64_t q = bid.x * int64_t(blockDim.x) + threadIdx.x; q < (n); q += int64_t(gd.x) * blockDim.x)

struct CastA { const double* a; float* b; int64_t n; };
__device__ __forceinline__ void cast_d2f_body(const uint3 bid, const uint3 gd, const double* __restrict__ a,
                                              float* __restrict__ b, int64_t n) {
  HHG_GRID_LOOP(q, n) b[q] = float(a[q]);
}
__global__ void k_cast_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  cast_d2f_body(blockIdx, gridDim, a, b, n);
}
__global__ void kb_cast_d2f(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<CastA>(items, n, bid, gd);
  cast_d2f_body(bid, gd, it.a.a, it.a.b, it.a.n);
}
struct AddF2dA { const float* a; double* b; int64_t n; };
__device__ __forceinline__ void add_f2d_body(const uint3 bid, const uint3 gd, const float* __restrict__ a,
                                             double* __restrict__ b, int64_t n) {
  HHG_GRID_LOOP(q, n) b[q] += double(a[q]);
}
__global__ void k_add_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  add_f2d_body(blockIdx, gridDim, a, b, n);
}
__global__ void kb_add_f2d(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<AddF2dA>(items, n, bid, gd);
  add_f2d_body(bid, gd, it.a.a, it.a.b, it.a.n);
}
// zero n 4-byte words
struct ZeroA { unsigned* p; int64_t n; };
__device__ __forceinline__ void zero_body(const uint3 bid, const uint3 gd, unsigned* __restrict__ p, int64_t n) {
  HHG_GRID_LOOP(q, n) p[q] = 0u;
}
__global__ void kb_zero(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<ZeroA>(items, n, bid, gd);
  zero_body(bid, gd, it.a.p, it.a.n);
}
template <class T>
__global__ void k_axpy(T alpha, const T* __restrict__ x, T* __restrict__ y, int64_t n) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x)
    y[q] += alpha * x[q];
}
template <class T>
struct XpbyA { const T* x; T beta; const T* y; T* z; int64_t n; };
template <class T>
__device__ __forceinline__ void xpby_body(const uint3 bid, const uint3 gd, const T* __restrict__ x, T beta,
                                          const T* __restrict__ y, T* __restrict__ z, int64_t n) {
  HHG_GRID_LOOP(q, n) z[q] = x[q] + beta * y[q];
}
template <class T>
__global__ void k_xpby(const T* __restrict__ x, T beta, const T* __restrict__ y, T* __restrict__ z, int64_t n) {
  xpby_body<T>(blockIdx, gridDim, x, beta, y, z, n);
}
template <class T>
__global__ void kb_xpby(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<XpbyA<T>>(items, n, bid, gd);
  xpby_body<T>(bid, gd, it.a.x, it.a.beta, it.a.y, it.a.z, it.a.n);
}
__global__ void k_inv(const double* __restrict__ a, double* __restrict__ b, int64_t n) {
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < n; q += int64_t(gridDim.x) * blockDim.x)
    b[q] = a[q] != 0.0 ? 1.0 / a[q] : 0.0;
}

inline int lin_blocks(int64_t n) { return int(std::min<int64_t>((n + 255) / 256, 152 * 8)); }

}  // namespace

// ============================================================ host wrappers
// While a batch records (g_rec set), each wrapper records its launch instead:
// a work item of the batched kernel, or (kernels without one) the launch itself.
#define HHG_NATIVE(...)                                                   \
  if (g_rec) {                                                            \
    g_rec->native([=](cudaStream_t s_) { __VA_ARGS__; });                 \
    return;                                                               \
  }
#define HHG_BATCHED(fn, grd, blk, A, ...)                                                                   \
  if (g_rec) {                                                                                             \
    g_rec->add(reinterpret_cast<const void*>(fn), grd, blk, 0, 1, A{__VA_ARGS__});                        \
    return;                                                                                                \
  }

template <class T>
void launch_apply(const Geo& g, const OpDev& op, int mode, const T* x, const T* b, T* y, double alpha,
                  cudaStream_t s) {
  HHG_NATIVE(launch_apply<T>(g, op, mode, x, b, y, alpha, s_))
  dim3 blk(32, 4, 1);
  if (op.nrows == 0) return;
  dim3 grd((g.nx + 1 + 31) / 32, (g.ny + 1 + 3) / 4, (g.nz + 1) * op.nrows);
  ++g_launches;
  if (mode == MODE_SET) k_apply<T, MODE_SET><<<grd, blk, 0, s>>>(g, op, x, b, y, T(alpha));
  else if (mode == MODE_RES) k_apply<T, MODE_RES><<<grd, blk, 0, s>>>(g, op, x, b, y, T(alpha));
  else k_apply<T, MODE_ADD><<<grd, blk, 0, s>>>(g, op, x, b, y, T(alpha));
}

template <class T>
void launch_apply_shell(const Geo& g, const OpDev& op, int mode, const T* x, const T* b, T* y, double alpha,
                        cudaStream_t s) {
  HHG_NATIVE(launch_apply_shell<T>(g, op, mode, x, b, y, alpha, s_))
  if (op.nrows == 0) return;
  if (g.nx < 4 || g.ny < 4 || g.nz < 4) return launch_apply<T>(g, op, mode, x, b, y, alpha, s);
  auto go = [&](int inner) {
    const int64_t n = inner ? 4 * int64_t(g.nx + 1) + 4 * int64_t(g.ny - 3) : int64_t(g.nx + 1) * (g.ny + 1);
    const int np = inner ? g.nz - 3 : 4;
    dim3 grd(unsigned((n + 127) / 128), unsigned(np * op.nrows), 1);
    ++g_launches;
    if (mode == MODE_SET) k_apply_shell<T, MODE_SET><<<grd, 128, 0, s>>>(g, op, inner, x, b, y, T(alpha));
    else if (mode == MODE_RES) k_apply_shell<T, MODE_RES><<<grd, 128, 0, s>>>(g, op, inner, x, b, y, T(alpha));
    else k_apply_shell<T, MODE_ADD><<<grd, 128, 0, s>>>(g, op, inner, x, b, y, T(alpha));
  };
  go(0);
  go(1);
}

template <class T>
void launch_gs(const Geo& g, const OpDev& A, int grp, int colour, double inv_diag, T* u, const T* rhs,
               cudaStream_t s) {
  HHG_NATIVE(launch_gs<T>(g, A, grp, colour, inv_diag, u, rhs, s_))
  dim3 blk(32, 4, 1);
  const int ni = colour >= 0 ? (g.nx + 1 + 3) / 4 : g.nx + 1;
  dim3 grd((ni + 31) / 32, (g.ny + 1 + 3) / 4, g.nz + 1);
  ++g_launches;
  k_gs<T><<<grd, blk, 0, s>>>(g, A, grp, colour, T(inv_diag), u, rhs);
}

template <class T>
void launch_pupdate(const Geo& g, T* p, const T* r, const double* inv_mlhat, double inv_omega_inv, cudaStream_t s) {
  dim3 blk(32, 4, 1);
  dim3 grd((g.nx + 1 + 31) / 32, (g.ny + 1 + 3) / 4, g.nz + 1);
  HHG_BATCHED(kb_pupdate<T>, grd, blk, PUpdateA<T>, g, p, r, inv_mlhat, inv_omega_inv)
  ++g_launches;
  k_pupdate<T><<<grd, blk, 0, s>>>(g, p, r, inv_mlhat, inv_omega_inv);
}

template <class T>
void launch_sub_scalar_p(const Geo& g, T* p, const double* sum, double scale, cudaStream_t s) {
  dim3 blk(32, 4, 1);
  dim3 grd((g.nx + 1 + 31) / 32, (g.ny + 1 + 3) / 4, g.nz + 1);
  HHG_BATCHED(kb_sub_scalar_p<T>, grd, blk, SubScalarA<T>, g, p, sum, scale)
  ++g_launches;
  k_sub_scalar_p<T><<<grd, blk, 0, s>>>(g, p, sum, scale);
}

template <class T>
void launch_prolong(const Geo& gf, const Geo& gc, const XferDev& X, int base_f, int base_c, int ncomp, int G,
                    bool interior_only, const T* xc, T* xf, cudaStream_t s) {
  dim3 blk(32, 4, 1);
  dim3 grd((gf.nx + 1 + 31) / 32, (gf.ny + 1 + 3) / 4, (gf.nz + 1) * G);
  HHG_BATCHED(kb_prolong<T>, grd, blk, XferA<T>, gf, gc, X, base_f, base_c, ncomp, G, interior_only ? 1 : 0, xc, xf)
  ++g_launches;
  k_prolong<T><<<grd, blk, 0, s>>>(gf, gc, X, base_f, base_c, ncomp, G, interior_only ? 1 : 0, xc, xf);
}

template <class T>
void launch_restrict(const Geo& gf, const Geo& gc, const XferDev& X, int base_f, int base_c, int ncomp, int G,
                     bool interior_only, const T* rf, T* rc, cudaStream_t s) {
  // lanes per coarse DoF: about eight terms each
  const int P = X.rmax > 32 ? 8 : X.rmax > 16 ? 4 : X.rmax > 8 ? 2 : 1;
  dim3 blk(128, 1, 1);
  dim3 grd((gc.nx + 1 + 128 / P - 1) / (128 / P), gc.ny + 1, (gc.nz + 1) * G);
  const int io = interior_only ? 1 : 0;
  if (g_rec) {
    const void* fn = P == 8   ? reinterpret_cast<const void*>(kb_restrict<T, 8>)
                     : P == 4 ? reinterpret_cast<const void*>(kb_restrict<T, 4>)
                     : P == 2 ? reinterpret_cast<const void*>(kb_restrict<T, 2>)
                              : reinterpret_cast<const void*>(kb_restrict<T, 1>);
    g_rec->add(fn, grd, blk, 0, 1, XferA<T>{gf, gc, X, base_f, base_c, ncomp, G, io, rf, rc});
    return;
  }
  ++g_launches;
  switch (P) {
    case 8: k_restrict<T, 8><<<grd, blk, 0, s>>>(gf, gc, X, base_f, base_c, ncomp, G, io, rf, rc); break;
    case 4: k_restrict<T, 4><<<grd, blk, 0, s>>>(gf, gc, X, base_f, base_c, ncomp, G, io, rf, rc); break;
    case 2: k_restrict<T, 2><<<grd, blk, 0, s>>>(gf, gc, X, base_f, base_c, ncomp, G, io, rf, rc); break;
    default: k_restrict<T, 1><<<grd, blk, 0, s>>>(gf, gc, X, base_f, base_c, ncomp, G, io, rf, rc); break;
  }
}

template <class T>
void launch_reduce(int mode, const T* a, const T* b, const double* w, int64_t n, double* partials, int max_blocks,
                   double* out, cudaStream_t s) {
  int nb = int(std::min<int64_t>((n + 255) / 256, max_blocks));
  if (nb < 1) nb = 1;
  if (g_rec) {
    const void* fn = mode == RED_SQ     ? reinterpret_cast<const void*>(kb_reduce_partial<T, RED_SQ>)
                     : mode == RED_DOT  ? reinterpret_cast<const void*>(kb_reduce_partial<T, RED_DOT>)
                     : mode == RED_WSUM ? reinterpret_cast<const void*>(kb_reduce_partial<T, RED_WSUM>)
                                        : reinterpret_cast<const void*>(kb_reduce_partial<T, RED_SUM>);
    g_rec->add(fn, dim3(nb), dim3(256), 0, 1, ReduceA<T>{a, b, w, n, partials});
    g_rec->add(reinterpret_cast<const void*>(kb_reduce_final), dim3(1), dim3(256), 0, 1, FinalA{partials, nb, out});
    return;
  }
  g_launches += 2;
  switch (mode) {
    case RED_SQ: k_reduce_partial<T, RED_SQ><<<nb, 256, 0, s>>>(a, b, w, n, partials); break;
    case RED_DOT: k_reduce_partial<T, RED_DOT><<<nb, 256, 0, s>>>(a, b, w, n, partials); break;
    case RED_WSUM: k_reduce_partial<T, RED_WSUM><<<nb, 256, 0, s>>>(a, b, w, n, partials); break;
    default: k_reduce_partial<T, RED_SUM><<<nb, 256, 0, s>>>(a, b, w, n, partials); break;
  }
  k_reduce_final<<<1, 256, 0, s>>>(partials, nb, out);
}

template <class T>
void launch_canon_scatter(const Geo& g, const double* src, T* dst, int64_t nvn, int64_t npn, bool with_pressure,
                          bool boundary_only, cudaStream_t s) {
  HHG_NATIVE(launch_canon_scatter<T>(g, src, dst, nvn, npn, with_pressure, boundary_only, s_))
  ++g_launches;
  dim3 grd(unsigned(std::min<int64_t>((nvn + 255) / 256, 152 * 8)), with_pressure ? 4 : 3);
  k_canon_scatter<T><<<grd, 256, 0, s>>>(g, src, dst, nvn, npn, boundary_only ? 1 : 0);
}

template <class T>
void launch_canon_gather(const Geo& g, const T* src, double* dst, int64_t nvn, int64_t npn, cudaStream_t s) {
  HHG_NATIVE(launch_canon_gather<T>(g, src, dst, nvn, npn, s_))
  ++g_launches;
  dim3 grd(unsigned(std::min<int64_t>((nvn + 255) / 256, 152 * 8)), 4);
  k_canon_gather<T><<<grd, 256, 0, s>>>(g, src, dst, nvn, npn);
}

template <class T>
void launch_coarse(const double* Z, int n, const int64_t* idx, const T* b, T* x, cudaStream_t s) {
  HHG_BATCHED(kb_coarse<T>, dim3(n), dim3(128), CoarseA<T>, Z, n, idx, b, x)
  ++g_launches;
  k_coarse<T><<<n, 128, 0, s>>>(Z, n, idx, b, x);
}

void launch_cast_d2f(const double* a, float* b, int64_t n, cudaStream_t s) {
  HHG_BATCHED(kb_cast_d2f, dim3(lin_blocks(n)), dim3(256), CastA, a, b, n)
  ++g_launches;
  k_cast_d2f<<<lin_blocks(n), 256, 0, s>>>(a, b, n);
}
void launch_add_f2d(const float* a, double* b, int64_t n, cudaStream_t s) {
  HHG_BATCHED(kb_add_f2d, dim3(lin_blocks(n)), dim3(256), AddF2dA, a, b, n)
  ++g_launches;
  k_add_f2d<<<lin_blocks(n), 256, 0, s>>>(a, b, n);
}
template <class T>
void launch_axpy(double alpha, const T* x, T* y, int64_t n, cudaStream_t s) {
  HHG_NATIVE(launch_axpy<T>(alpha, x, y, n, s_))
  ++g_launches;
  k_axpy<T><<<lin_blocks(n), 256, 0, s>>>(T(alpha), x, y, n);
}
template <class T>
void launch_xpby(const T* x, double beta, const T* y, T* z, int64_t n, cudaStream_t s) {
  HHG_BATCHED(kb_xpby<T>, dim3(lin_blocks(n)), dim3(256), XpbyA<T>, x, T(beta), y, z, n)
  ++g_launches;
  k_xpby<T><<<lin_blocks(n), 256, 0, s>>>(x, T(beta), y, z, n);
}
void launch_inv(const double* a, double* b, int64_t n, cudaStream_t s) {
  HHG_NATIVE(launch_inv(a, b, n, s_))
  ++g_launches;
  k_inv<<<lin_blocks(n), 256, 0, s>>>(a, b, n);
}

cudaError_t launch_zero(void* p, size_t bytes, cudaStream_t s) {
  if (g_rec) {
    const int64_t words = int64_t(bytes / 4);
    g_rec->add(reinterpret_cast<const void*>(kb_zero), dim3(lin_blocks(words)), dim3(256), 0, 1,
               ZeroA{static_cast<unsigned*>(p), words}, 0);
    return cudaSuccess;
  }
  return cudaMemsetAsync(p, 0, bytes, s);
}

template void launch_canon_scatter<double>(const Geo&, const double*, double*, int64_t, int64_t, bool, bool, cudaStream_t);
template void launch_canon_scatter<float>(const Geo&, const double*, float*, int64_t, int64_t, bool, bool, cudaStream_t);
template void launch_canon_gather<double>(const Geo&, const double*, double*, int64_t, int64_t, cudaStream_t);
template void launch_canon_gather<float>(const Geo&, const float*, double*, int64_t, int64_t, cudaStream_t);

#define HHG_INST(T)                                                                                              \
  template void launch_apply<T>(const Geo&, const OpDev&, int, const T*, const T*, T*, double, cudaStream_t);     \
  template void launch_apply_shell<T>(const Geo&, const OpDev&, int, const T*, const T*, T*, double,              \
                                      cudaStream_t);                                                              \
  template void launch_gs<T>(const Geo&, const OpDev&, int, int, double, T*, const T*, cudaStream_t);              \
  template void launch_pupdate<T>(const Geo&, T*, const T*, const double*, double, cudaStream_t);                 \
  template void launch_sub_scalar_p<T>(const Geo&, T*, const double*, double, cudaStream_t);                      \
  template void launch_prolong<T>(const Geo&, const Geo&, const XferDev&, int, int, int, int, bool, const T*, T*, \
                                  cudaStream_t);                                                                  \
  template void launch_restrict<T>(const Geo&, const Geo&, const XferDev&, int, int, int, int, bool, const T*,    \
                                   T*, cudaStream_t);                                                             \
  template void launch_reduce<T>(int, const T*, const T*, const double*, int64_t, double*, int, double*,          \
                                 cudaStream_t);                                                                   \
  template void launch_coarse<T>(const double*, int, const int64_t*, const T*, T*, cudaStream_t);                 \
  template void launch_axpy<T>(double, const T*, T*, int64_t, cudaStream_t);                                      \
  template void launch_xpby<T>(const T*, double, const T*, T*, int64_t, cudaStream_t);
HHG_INST(double)
HHG_INST(float)

}  // namespace hhg
