// Specialised stencil kernels for the hot operators of the V-cycle:
// the Gauss-Seidel phases of the inexact Uzawa velocity step, and the
// FULL / B^T / (B, -C) row evaluations (apply or residual mode).
//
// Inputs must have zero Dirichlet velocity entries (the lifting form used by
// the solver): boundary pressure rows then use the merged B stencil.
//
// The term count of every row is a compile-time constant (generated at build
// time from the stencil builder, structure.inc), so each row is one fully
// unrolled sequence of independent loads and FMAs.  The weights and the
// linear offsets of the level (array * array_stride + di + dj*sx + dk*sy) are
// __grid_constant__ kernel parameters: every term reads its weight and offset
// from the constant bank, not from memory.  Rows on the domain boundary
// (pressure rows of the box faces) take the per-cube path of the generic
// tables; Dirichlet velocity rows are zero.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "batch.h"
#include "fast.h"
#include "kernels.h"
#include "structure.inc"

namespace hhg {
namespace {

__device__ __forceinline__ int64_t fsite(const Geo& g, int i, int j, int k) {
  return int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy;
}

template <class T> __device__ __forceinline__ T bw(const OpDev& op, int t);
template <> __device__ __forceinline__ double bw<double>(const OpDev& op, int t) { return __ldg(op.bw64 + t); }
template <> __device__ __forceinline__ float bw<float>(const OpDev& op, int t) { return __ldg(op.bw32 + t); }

// per-cube evaluation of a boundary row r of the generic tables: returns the
// three segment sums
template <class T>
__device__ __forceinline__ void boundary_row(const Geo& g, const OpDev& op, int r, int i, int j, int k, const T* x,
                                          int64_t idx, T& s0, T& s1, T& s2) {
  const DRow row = op.rows[r];
  int t = row.b0;
  const int ms[3] = {row.m0, row.m1, row.m2};
  T acc[3] = {T(0), T(0), T(0)};
  for (int s = 0; s < 3; ++s) {
    T a = T(0);
    for (int e = 0; e < ms[s]; ++e, ++t) {
      const DTermB tm = op.bterms[t];
      const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
      if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
      a += bw<T>(op, t) * x[int64_t(tm.arr) * g.arr + idx + tm.off];
    }
    acc[s] = a;
  }
  s0 = acc[0]; s1 = acc[1]; s2 = acc[2];
}

// per-cube evaluation of the third segment (C terms) of a boundary row
template <class T>
__device__ __forceinline__ T boundary_seg2(const Geo& g, const OpDev& op, int r, int i, int j, int k, const T* x,
                                           int64_t idx) {
  const DRow row = op.rows[r];
  T a = T(0);
  for (int t = row.b0 + row.m0 + row.m1; t < row.b0 + row.m0 + row.m1 + row.m2; ++t) {
    const DTermB tm = op.bterms[t];
    const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
    if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
    a += bw<T>(op, t) * x[int64_t(tm.arr) * g.arr + idx + tm.off];
  }
  return a;
}

template <class S, int R, class F>
__device__ __forceinline__ void dispatch(int r, F&& f) {
  if constexpr (R < S::R) {
    if (r == R) f(std::integral_constant<int, R>{});
    else dispatch<S, R + 1>(r, f);
  }
}

// sum of w[t] * xs[off[t]] for t in [T0, T0 + N): one fully unrolled chain
template <int T0, int N, class T, class Tab>
__device__ __forceinline__ T seg_sum(const Tab& tab, const T* __restrict__ xs) {
  T a = T(0);
#pragma unroll
  for (int t = 0; t < N; ++t) a += tab.w[T0 + t] * __ldg(xs + tab.off[T0 + t]);
  return a;
}

// the same sums at V sites 32 apart (xs + 32 v): per term one address and V
// loads at compile-time distances
template <int T0, int N, int V, class T, class Tab>
__device__ __forceinline__ void seg_sum_v(const Tab& tab, const T* __restrict__ xs, T (&a)[V]) {
#pragma unroll
  for (int v = 0; v < V; ++v) a[v] = T(0);
#pragma unroll
  for (int t = 0; t < N; ++t) {
    const T wt = tab.w[T0 + t];
    const T* p = xs + tab.off[T0 + t];
#pragma unroll
    for (int v = 0; v < V; ++v) a[v] += wt * __ldg(p + 32 * v);
  }
}

// launch shapes (threads per block, k planes per thread, sites per thread)
// are run-time parameters chosen per level by the autotuner (hhg_autotune)

// ------------------------------------------------------------- row kernels
// one row at site (i, j, k); bij: the site lies on an i or j face of the box
template <int VARNU, class T, int MODE, int OUT, int OG, int ALL, int T0, int N0, int N1, int N2, class Tab>
__device__ __forceinline__ void row_site(const Geo& g, int R, int i, int j, int k, bool bij, const T* __restrict__ x,
                                         const T* __restrict__ b, T* __restrict__ y, T alpha, const OpDev& op,
                                         const Tab& tab) {
  constexpr int oz = OG == 3 || OG == 5 || OG == 6 || OG == 7;
  const int64_t idx = fsite(g, i, j, k);
  T* yo = y + int64_t(OUT) * g.arr + idx;
  const bool bnd = bij || 2 * k + oz == 0 || 2 * k + oz == 2 * g.nz;
  T a0, a1, a2;
  if (!bnd) {
    const T* xs = x + idx;
    a0 = seg_sum<T0, N0, T>(tab, xs);
    a1 = seg_sum<T0 + N0, N1, T>(tab, xs);
    a2 = seg_sum<T0 + N0 + N1, N2, T>(tab, xs);
  } else if (ALL) {
    // boundary pressure row: with zero Dirichlet velocity entries the merged
    // B terms are exact (every tetrahedron containing an interior velocity
    // DoF lies inside the domain; boundary and halo velocity values are 0);
    // only the C terms need the per-cube restriction to the domain
    const T* xs = x + idx;
    a0 = seg_sum<T0, N0, T>(tab, xs);
    a1 = seg_sum<T0 + N0, N1, T>(tab, xs);
    a2 = N2 > 0 ? boundary_seg2<T>(g, op, R, i, j, k, x, idx) : T(0);
  } else {
    if (MODE != MODE_ADD) *yo = T(0);
    return;
  }
  T v = a0;
  if (VARNU) {
    v += T(g.esc[k]) * a1 + T(g.eisc[k]) * a2;
  } else {
    v += a1 + a2;
  }
  if (MODE == MODE_SET) *yo = v;
  else if (MODE == MODE_RES) *yo = b[int64_t(OUT) * g.arr + idx] - v;
  else *yo += alpha * v;
}

// grid: x over the (i, j) plane of sites (flat, i fastest), y = groups of
// kp planes, z = row.  The row is the slowest grid dimension, so the
// blocks resident at the same time run the same (fully unrolled) row code.
template <int DISC, int VARNU, int OP, class T, int MODE, int OUT, int OG, int ALL, int T0, int N0, int N1, int N2,
          class Tab>
__device__ __forceinline__ void eval_row(const uint3 bid, const Geo& g, int R, const T* __restrict__ x,
                                         const T* __restrict__ b, T* __restrict__ y, T alpha, const OpDev& op,
                                         const Tab& tab, int kp) {
  constexpr int ox = OG == 1 || OG == 4 || OG == 5 || OG == 7;
  constexpr int oy = OG == 2 || OG == 4 || OG == 6 || OG == 7;
  constexpr int oz = OG == 3 || OG == 5 || OG == 6 || OG == 7;
  const int w = g.nx + 1 - ox;                       // sites per i row of this group
  const int q = bid.x * blockDim.x + threadIdx.x;
  const int j = q / w;
  const int i = q - j * w;
  if (j > g.ny - oy) return;
  const int k0 = bid.y * kp;
  const bool bij = 2 * i + ox == 0 || 2 * i + ox == 2 * g.nx || 2 * j + oy == 0 || 2 * j + oy == 2 * g.ny;
#pragma unroll 1
  for (int k = k0; k < k0 + kp && k <= g.nz - oz; ++k)
    row_site<VARNU, T, MODE, OUT, OG, ALL, T0, N0, N1, N2>(g, R, i, j, k, bij, x, b, y, alpha, op, tab);
}

// V sites per thread: a warp takes V runs of 32 consecutive positions
// m = i + j sx of the padded (i, j) plane (lane l: m0 + l + 32 v).  The site
// index is m + 1 + sx + (k+1) sy, so the V sites of a term are V coalesced
// loads at fixed distances from one address.  Positions in the row padding
// (i > nx - ox) are evaluated but not stored (their reads stay inside the
// plane's halo rows); a warp whose last run passes the group's last site
// evaluates its sites one by one (its runs would read past the plane).
template <int DISC, int VARNU, int OP, class T, int MODE, int V, int OUT, int OG, int ALL, int T0, int N0, int N1,
          int N2, class Tab>
__device__ __forceinline__ void eval_row_vec(const uint3 bid, const Geo& g, int R, const T* __restrict__ x,
                                             const T* __restrict__ b, T* __restrict__ y, T alpha, const OpDev& op,
                                             const Tab& tab, int kp) {
  constexpr int ox = OG == 1 || OG == 4 || OG == 5 || OG == 7;
  constexpr int oy = OG == 2 || OG == 4 || OG == 6 || OG == 7;
  constexpr int oz = OG == 3 || OG == 5 || OG == 6 || OG == 7;
  const int m0 = ((bid.x * blockDim.x + threadIdx.x) >> 5) * (32 * V);
  const int lane = int(threadIdx.x & 31);
  const int mlast = (g.ny - oy) * g.sx + (g.nx - ox);   // position of the group's last site in the plane
  if (m0 > mlast) return;
  const int k0 = bid.y * kp, k1 = min(k0 + kp, g.nz - oz + 1);
  if (m0 + 32 * V - 1 > mlast) {                     // warp-uniform: the plane's last warp
#pragma unroll 1
    for (int k = k0; k < k1; ++k)
#pragma unroll 1
      for (int v = 0; v < V; ++v) {
        const int m = m0 + lane + 32 * v;
        const int j = m / g.sx, i = m - j * g.sx;
        if (m > mlast || i > g.nx - ox) continue;
        const bool bij = 2 * i + ox == 0 || 2 * i + ox == 2 * g.nx || 2 * j + oy == 0 || 2 * j + oy == 2 * g.ny;
        row_site<VARNU, T, MODE, OUT, OG, ALL, T0, N0, N1, N2>(g, R, i, j, k, bij, x, b, y, alpha, op, tab);
      }
    return;
  }
  int iv[V], jv[V];
  bool okv[V], bijv[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const int m = m0 + lane + 32 * v;
    jv[v] = m / g.sx;
    iv[v] = m - jv[v] * g.sx;
    okv[v] = iv[v] <= g.nx - ox;
    bijv[v] = 2 * iv[v] + ox == 0 || 2 * iv[v] + ox == 2 * g.nx || 2 * jv[v] + oy == 0 || 2 * jv[v] + oy == 2 * g.ny;
  }
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const int64_t idx = int64_t(m0 + lane) + 1 + g.sx + int64_t(k + 1) * g.sy;
    const T* xs = x + idx;
    T a0[V], a1[V], a2[V];
    seg_sum_v<T0, N0, V>(tab, xs, a0);
    seg_sum_v<T0 + N0, N1, V>(tab, xs, a1);
    seg_sum_v<T0 + N0 + N1, N2, V>(tab, xs, a2);
    const bool bk = 2 * k + oz == 0 || 2 * k + oz == 2 * g.nz;
    T es = T(1), eis = T(1);
    if (VARNU) {
      es = T(g.esc[k]);
      eis = T(g.eisc[k]);
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      if (!okv[v]) continue;
      const bool bnd = bijv[v] || bk;
      const int64_t iy = int64_t(OUT) * g.arr + idx + 32 * v;
      if (bnd && !ALL) {                             // Dirichlet velocity row
        if (MODE != MODE_ADD) y[iy] = T(0);
        continue;
      }
      T s2 = a2[v];
      if (N2 > 0 && bnd) s2 = boundary_seg2<T>(g, op, R, iv[v], jv[v], k, x, idx + 32 * v);
      T val = a0[v];
      if (VARNU) {
        val += es * a1[v] + eis * s2;
      } else {
        val += a1[v] + s2;
      }
      if (MODE == MODE_SET) y[iy] = val;
      else if (MODE == MODE_RES) y[iy] = b[iy] - val;
      else y[iy] += alpha * val;
    }
  }
}

// Programmatic dependent launch (Gauss-Seidel phases): a kernel launched with
// the programmatic-serialization attribute may start while its predecessor in
// the stream finishes; it waits here until the predecessor has completed and
// its writes are visible (no-op for an ordinary launch), and each block
// signals its own successor once its work is done.  (In the stencil-row
// kernels the wait doubles the register count of the 25-way row dispatch, so
// those launch plainly.)
__device__ __forceinline__ void pdl_wait() { cudaGridDependencySynchronize(); }
__device__ __forceinline__ void pdl_trigger() { cudaTriggerProgrammaticLaunchCompletion(); }

// FP32 P2-P1 rows: at most 80 registers (three 256-thread blocks per SM);
// the shorter P1-P1 rows, and FP64 (bound by its arithmetic), uncapped
// the work item's table (a device copy) staged in the block's shared memory,
// so that the unrolled terms read their weights and offsets from there
template <class Tab>
__device__ __forceinline__ const Tab& stage_table(const Tab* src) {
  extern __shared__ __align__(16) unsigned char kb_tab_smem[];
  static_assert(sizeof(Tab) % 4 == 0, "tables are copied as 4-byte words");
  const unsigned* s = reinterpret_cast<const unsigned*>(src);
  unsigned* d = reinterpret_cast<unsigned*>(kb_tab_smem);
  for (int q = threadIdx.x; q < int(sizeof(Tab) / 4); q += blockDim.x) d[q] = __ldg(s + q);
  __syncthreads();
  return *reinterpret_cast<const Tab*>(kb_tab_smem);
}

// arguments of the row kernels as a work item of a merged launch (the table
// as a device copy)
template <class T, class Tab>
struct RowsA { Geo g; const T* x; const T* b; T* y; T alpha; OpDev op; int kp; const Tab* tab; };

template <int DISC, int VARNU, int OP, class T, int MODE, int V, class Tab>
__device__ __forceinline__ void rows_vec_body(const uint3 bid, const Geo& g, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ y, T alpha, const OpDev& op,
                                              int kp, const Tab& tab) {
  using S = gen::S<DISC, VARNU, OP>;
  dispatch<S, 0>(int(bid.z), [&](auto rc) {
    constexpr int R = decltype(rc)::value;
    constexpr gen::RowS rw = S::rows[R];
    eval_row_vec<DISC, VARNU, OP, T, MODE, V, rw.out, rw.og, rw.all, rw.t0, rw.n0, rw.n1, rw.n2>(bid, g, R, x, b, y,
                                                                                                alpha, op, tab, kp);
  });
}
template <int DISC, int VARNU, int OP, class T, int MODE, int V>
__global__ void __launch_bounds__(256, DISC == 2 && sizeof(T) == 4 ? 3 : 1)
    k_rows_vec(Geo g, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y, T alpha, OpDev op, int kp,
               const __grid_constant__ FastTab<T, gen::S<DISC, VARNU, OP>::N> tab) {
  rows_vec_body<DISC, VARNU, OP, T, MODE, V>(blockIdx, g, x, b, y, alpha, op, kp, tab);
}
template <int DISC, int VARNU, int OP, class T, int MODE, int V>
__global__ void __launch_bounds__(256, DISC == 2 && sizeof(T) == 4 ? 3 : 1) kb_rows_vec(const void* items, int n) {
  using Tab = FastTab<T, gen::S<DISC, VARNU, OP>::N>;
  uint3 bid, gd;
  const auto& it = batch_item<RowsA<T, Tab>>(items, n, bid, gd);
  const RowsA<T, Tab>& a = it.a;
  const Tab& tab = stage_table(a.tab);
  rows_vec_body<DISC, VARNU, OP, T, MODE, V>(bid, a.g, a.x, a.b, a.y, a.alpha, a.op, a.kp, tab);
}

template <int DISC, int VARNU, int OP, class T, int MODE, class Tab>
__device__ __forceinline__ void rows_fast_body(const uint3 bid, const Geo& g, const T* __restrict__ x,
                                               const T* __restrict__ b, T* __restrict__ y, T alpha, const OpDev& op,
                                               int kp, const Tab& tab) {
  using S = gen::S<DISC, VARNU, OP>;
  dispatch<S, 0>(int(bid.z), [&](auto rc) {
    constexpr int R = decltype(rc)::value;
    constexpr gen::RowS rw = S::rows[R];
    eval_row<DISC, VARNU, OP, T, MODE, rw.out, rw.og, rw.all, rw.t0, rw.n0, rw.n1, rw.n2>(bid, g, R, x, b, y, alpha,
                                                                                          op, tab, kp);
  });
}
template <int DISC, int VARNU, int OP, class T, int MODE>
__global__ void __launch_bounds__(256)
    k_rows_fast(Geo g, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y, T alpha, OpDev op, int kp,
                const __grid_constant__ FastTab<T, gen::S<DISC, VARNU, OP>::N> tab) {
  rows_fast_body<DISC, VARNU, OP, T, MODE>(blockIdx, g, x, b, y, alpha, op, kp, tab);
}
template <int DISC, int VARNU, int OP, class T, int MODE>
__global__ void __launch_bounds__(256) kb_rows_fast(const void* items, int n) {
  using Tab = FastTab<T, gen::S<DISC, VARNU, OP>::N>;
  uint3 bid, gd;
  const auto& it = batch_item<RowsA<T, Tab>>(items, n, bid, gd);
  const RowsA<T, Tab>& a = it.a;
  const Tab& tab = stage_table(a.tab);
  rows_fast_body<DISC, VARNU, OP, T, MODE>(bid, a.g, a.x, a.b, a.y, a.alpha, a.op, a.kp, tab);
}

// -------------------------------------------------- Gauss-Seidel phase kernel
// sum over the 2^LP lanes of a group of consecutive lanes (all lanes of the
// warp take part)
template <int LP, class T>
__device__ __forceinline__ T lane_sum(T v) {
#pragma unroll
  for (int m = (1 << LP) >> 1; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// grid: x over the (i', j) plane (i' = i, or i / 4 for a vertex colour) times
// 2^LP lanes per site, z = k.  With LP > 0 the lanes of a site take every
// 2^LP-th term and add their sums by shuffles: shorter dependent chains and
// more threads for the small levels, whose phases are latency-bound.
// NC = 3: the three velocity components at once (u, rhs: block vectors);
// NC = 1: one component (u, rhs point to that component's first group array)
template <int DISC, int VARNU, int GRP, class T, int LP, int NC, int T0, int N1, class Tab>
__device__ __forceinline__ void gs_site(const uint3 bid, const Geo& g, T* __restrict__ u, const T* __restrict__ rhs,
                                        T inv_diag, int colour, const Tab& tab) {
  constexpr int ox = GRP == 1 || GRP == 4 || GRP == 5 || GRP == 7;
  constexpr int oy = GRP == 2 || GRP == 4 || GRP == 6 || GRP == 7;
  constexpr int oz = GRP == 3 || GRP == 5 || GRP == 6 || GRP == 7;
  constexpr int P = 1 << LP;
  const int k = bid.z;
  const int w = colour >= 0 ? (g.nx + 1 + 3) / 4 : g.nx + 1 - ox;
  const int q = bid.x * blockDim.x + threadIdx.x;
  const int site = q >> LP, p = q & (P - 1);
  const int j = site / w;
  int i = site - j * w;
  if (colour >= 0) i = 4 * i + (((colour - j - k) % 4) + 4) % 4;
  const int Px = 2 * i + ox, Py = 2 * j + oy, Pz = 2 * k + oz;
  const bool ok = Px > 0 && Py > 0 && Pz > 0 && Px < 2 * g.nx && Py < 2 * g.ny && Pz < 2 * g.nz;
  if (LP == 0 && !ok) return;
  const int64_t idx = ok ? fsite(g, i, j, k) : 0;
  const int64_t cs = int64_t(g.G) * g.arr;
  const T* us = u + idx;
  T a0 = T(0), a1 = T(0), a2 = T(0);
  if constexpr (LP == 0) {
#pragma unroll
    for (int t = 1; t < N1; ++t) {             // the diagonal is the first term
      const T wt = tab.w[T0 + t];
      const int o = tab.off[T0 + t];
      a0 += wt * us[o];
      if (NC == 3) {
        a1 += wt * us[o + cs];
        a2 += wt * us[o + 2 * cs];
      }
    }
  } else {
    if (ok) {
#pragma unroll
      for (int t0 = 1; t0 < N1; t0 += P) {
        const int t = t0 + p;
        if (t < N1) {
          const T wt = tab.w[T0 + t];
          const int o = tab.off[T0 + t];
          a0 += wt * us[o];
          if (NC == 3) {
            a1 += wt * us[o + cs];
            a2 += wt * us[o + 2 * cs];
          }
        }
      }
    }
    a0 = lane_sum<LP>(a0);                     // whole warps: the grid covers whole blocks
    if (NC == 3) {
      a1 = lane_sum<LP>(a1);
      a2 = lane_sum<LP>(a2);
    }
    if (!ok || p != 0) return;
  }
  T einv = T(1);
  if (VARNU) einv = T(g.eisc[k]);
  const int64_t o0 = int64_t(GRP) * g.arr + idx;
  u[o0] = (rhs[o0] * einv - a0) * inv_diag;
  if (NC == 3) {
    u[o0 + cs] = (rhs[o0 + cs] * einv - a1) * inv_diag;
    u[o0 + 2 * cs] = (rhs[o0 + 2 * cs] * einv - a2) * inv_diag;
  }
}

template <int DISC, int VARNU, int GRP, class T, int LP, int NC>
__global__ void __launch_bounds__(256)
    k_gs_fast(Geo g, T* __restrict__ u, const T* __restrict__ rhs, T inv_diag, int colour,
              const __grid_constant__ FastTab<T, gen::S<DISC, VARNU, OP_A>::N> tab) {
  using S = gen::S<DISC, VARNU, OP_A>;
  constexpr gen::RowS rw = S::rows[GRP];       // component-0 row of the group; all terms in segment 1
  static_assert(rw.n0 == 0 && rw.n2 == 0, "A rows carry only nu-scaled terms");
  pdl_wait();
  gs_site<DISC, VARNU, GRP, T, LP, NC, rw.t0, rw.n1>(blockIdx, g, u, rhs, inv_diag, colour, tab);
  pdl_trigger();
}
template <class T, class Tab>
struct GsA { Geo g; T* u; const T* rhs; T inv_diag; int colour; const Tab* tab; };
template <int DISC, int VARNU, int GRP, class T, int LP, int NC>
__global__ void __launch_bounds__(256) kb_gs_fast(const void* items, int n) {
  using S = gen::S<DISC, VARNU, OP_A>;
  using Tab = FastTab<T, S::N>;
  constexpr gen::RowS rw = S::rows[GRP];
  uint3 bid, gd;
  const auto& it = batch_item<GsA<T, Tab>>(items, n, bid, gd);
  const GsA<T, Tab>& a = it.a;
  const Tab& tab = stage_table(a.tab);
  gs_site<DISC, VARNU, GRP, T, LP, NC, rw.t0, rw.n1>(bid, a.g, a.u, a.rhs, a.inv_diag, a.colour, tab);
}

}  // namespace

// ================================================================= launchers
// Launches of at most about one wave (152 SMs x 8 blocks) may overlap their
// predecessor's tail (programmatic dependent launch): there the launch gap is
// a large part of the kernel time.  Longer grids are launched plainly.
constexpr int64_t kPdlMaxBlocks = 152 * 8;

template <class K, class... A>
void launch_pdl(K kernel, dim3 grd, dim3 blk, cudaStream_t s, A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grd;
  cfg.blockDim = blk;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = int64_t(grd.x) * grd.y * grd.z <= kPdlMaxBlocks ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, args...);
}

// launch geometry of the row kernels (plain launch and batch recording)
struct RowsGeo {
  dim3 grd, blk;
  int kp;
  bool vec;          // four sites per thread (k_rows_vec)
};
template <int DISC, int VARNU, int OP, class T>
RowsGeo rows_geo(const Geo& g, int mode, const Shape& sh) {
  using S = gen::S<DISC, VARNU, OP>;
  int nt = sh.row_threads, kp = sh.row_kplanes, sites = sizeof(T) == 8 ? sh.row_sites64 : sh.row_sites;
  if (OP == OP_BT && sh.bt_threads) {
    nt = sh.bt_threads; kp = sh.bt_kplanes; sites = sh.bt_sites;
  } else if (OP == OP_BC && sh.bc_threads) {
    nt = sh.bc_threads; kp = sh.bc_kplanes; sites = sh.bc_sites;
  }
  RowsGeo r;
  r.blk = dim3(nt, 1, 1);
  r.kp = kp;
  r.vec = sites == 4 && mode != MODE_ADD;
  if (r.vec) {
    // warps of 4 x 32 positions over the padded plane up to the last site
    const int64_t warps = ((int64_t(g.ny) * g.sx + g.nx + 1) + 127) / 128;
    r.grd = dim3(unsigned((warps * 32 + nt - 1) / nt), (g.nz + 1 + kp - 1) / kp, S::R);
  } else {
    const int plane = (g.nx + 1) * (g.ny + 1);
    r.grd = dim3((plane + nt - 1) / nt, (g.nz + 1 + kp - 1) / kp, S::R);
  }
  return r;
}

// launch geometry of a Gauss-Seidel phase
struct GsGeo {
  dim3 grd, blk;
  int lp;            // log2 of the lanes per site
};
inline GsGeo gs_geo(const Geo& g, int grp, int colour, const Shape& sh) {
  const int nt = grp == 0 && sh.gs_threads0 ? sh.gs_threads0 : sh.gs_threads;
  const int nl = grp == 0 ? sh.gs_lanes0 : sh.gs_lanes;
  GsGeo r;
  r.lp = nl == 4 ? 2 : nl == 2 ? 1 : 0;
  r.blk = dim3(nt, 1, 1);
  const int ni = colour >= 0 ? (g.nx + 1 + 3) / 4 : g.nx + 1;
  const int64_t plane = int64_t(ni) * (g.ny + 1) << r.lp;
  r.grd = dim3(unsigned((plane + nt - 1) / nt), 1, g.nz + 1);
  return r;
}

// the group and lane count of a phase as compile-time constants
template <class F>
void by_group_lanes(int grp, int lp, F&& f) {
  auto by_lanes = [&](auto gc) {
    if (lp == 2) f(gc, std::integral_constant<int, 2>{});
    else if (lp == 1) f(gc, std::integral_constant<int, 1>{});
    else f(gc, std::integral_constant<int, 0>{});
  };
  switch (grp) {
    case 0: by_lanes(std::integral_constant<int, 0>{}); break;
    case 1: by_lanes(std::integral_constant<int, 1>{}); break;
    case 2: by_lanes(std::integral_constant<int, 2>{}); break;
    case 3: by_lanes(std::integral_constant<int, 3>{}); break;
    case 4: by_lanes(std::integral_constant<int, 4>{}); break;
    case 5: by_lanes(std::integral_constant<int, 5>{}); break;
    case 6: by_lanes(std::integral_constant<int, 6>{}); break;
    case 7: by_lanes(std::integral_constant<int, 7>{}); break;
    default: break;
  }
}

#if defined(HHG_FAST_BATCHED)
// ------------------------------------------------ batch recording (kb_*)
template <int DISC, int VARNU, int OP, class T>
void record_rows(const Geo& g, const OpDev& op, const void* tab, int mode, const T* x, const T* b, T* y,
                 double alpha, const Shape& sh) {
  using Tab = FastTab<T, gen::S<DISC, VARNU, OP>::N>;
  const RowsGeo rg = rows_geo<DISC, VARNU, OP, T>(g, mode, sh);
  const Tab* dtab = static_cast<const Tab*>(g_rec->table(tab, sizeof(Tab)));
  const RowsA<T, Tab> ra{g, x, b, y, T(alpha), op, rg.kp, dtab};
  const void* fn;
  if (rg.vec)
    fn = mode == MODE_SET ? reinterpret_cast<const void*>(kb_rows_vec<DISC, VARNU, OP, T, MODE_SET, 4>)
                          : reinterpret_cast<const void*>(kb_rows_vec<DISC, VARNU, OP, T, MODE_RES, 4>);
  else
    fn = mode == MODE_SET   ? reinterpret_cast<const void*>(kb_rows_fast<DISC, VARNU, OP, T, MODE_SET>)
         : mode == MODE_RES ? reinterpret_cast<const void*>(kb_rows_fast<DISC, VARNU, OP, T, MODE_RES>)
                            : reinterpret_cast<const void*>(kb_rows_fast<DISC, VARNU, OP, T, MODE_ADD>);
  g_rec->add(fn, rg.grd, rg.blk, sizeof(Tab), 1, ra);
}

template <int DISC, int VARNU, class T>
void record_gs(const Geo& g, const void* tab, int grp, int colour, double inv_diag, T* u, const T* rhs,
               const Shape& sh, int comp) {
  using Tab = FastTab<T, gen::S<DISC, VARNU, OP_A>::N>;
  const GsGeo gg = gs_geo(g, grp, colour, sh);
  const Tab* dtab = static_cast<const Tab*>(g_rec->table(tab, sizeof(Tab)));
  const int64_t cs = comp < 0 ? 0 : int64_t(comp) * g.G * g.arr;   // the component's first group array
  by_group_lanes(grp, gg.lp, [&](auto gc, auto lc) {
    constexpr int GRP = decltype(gc)::value, LP = decltype(lc)::value;
    if constexpr (DISC == 2 || GRP == 0) {
      const void* fn = comp < 0 ? reinterpret_cast<const void*>(kb_gs_fast<DISC, VARNU, GRP, T, LP, 3>)
                                : reinterpret_cast<const void*>(kb_gs_fast<DISC, VARNU, GRP, T, LP, 1>);
      g_rec->add(fn, gg.grd, gg.blk, sizeof(Tab), 1, GsA<T, Tab>{g, u + cs, rhs + cs, T(inv_diag), colour, dtab});
    }
  });
}
#else
// ------------------------------------------------------- plain launches
template <int DISC, int VARNU, int OP, class T>
void launch_rows_fast(const Geo& g, const OpDev& op, const void* tab, int mode, const T* x, const T* b, T* y,
                      double alpha, const Shape& sh, cudaStream_t s) {
  using Tab = FastTab<T, gen::S<DISC, VARNU, OP>::N>;
  const Tab& tb = *static_cast<const Tab*>(tab);
  const RowsGeo rg = rows_geo<DISC, VARNU, OP, T>(g, mode, sh);
  const int kp = rg.kp;
  ++g_launches;
  if (rg.vec) {
    if (mode == MODE_SET)
      k_rows_vec<DISC, VARNU, OP, T, MODE_SET, 4><<<rg.grd, rg.blk, 0, s>>>(g, x, b, y, T(alpha), op, kp, tb);
    else
      k_rows_vec<DISC, VARNU, OP, T, MODE_RES, 4><<<rg.grd, rg.blk, 0, s>>>(g, x, b, y, T(alpha), op, kp, tb);
    return;
  }
  if (mode == MODE_SET)
    k_rows_fast<DISC, VARNU, OP, T, MODE_SET><<<rg.grd, rg.blk, 0, s>>>(g, x, b, y, T(alpha), op, kp, tb);
  else if (mode == MODE_RES)
    k_rows_fast<DISC, VARNU, OP, T, MODE_RES><<<rg.grd, rg.blk, 0, s>>>(g, x, b, y, T(alpha), op, kp, tb);
  else
    k_rows_fast<DISC, VARNU, OP, T, MODE_ADD><<<rg.grd, rg.blk, 0, s>>>(g, x, b, y, T(alpha), op, kp, tb);
}

template <int DISC, int VARNU, class T>
void launch_gs_fast(const Geo& g, const void* tab, int grp, int colour, double inv_diag, T* u, const T* rhs,
                    const Shape& sh, int comp, cudaStream_t s) {
  using Tab = FastTab<T, gen::S<DISC, VARNU, OP_A>::N>;
  const Tab& tb = *static_cast<const Tab*>(tab);
  const GsGeo gg = gs_geo(g, grp, colour, sh);
  ++g_launches;
  const int64_t cs = comp < 0 ? 0 : int64_t(comp) * g.G * g.arr;   // the component's first group array
  by_group_lanes(grp, gg.lp, [&](auto gc, auto lc) {
    constexpr int GRP = decltype(gc)::value, LP = decltype(lc)::value;
    if constexpr (DISC == 2 || GRP == 0) {
      if (comp < 0)
        launch_pdl(k_gs_fast<DISC, VARNU, GRP, T, LP, 3>, gg.grd, gg.blk, s, g, u, rhs, T(inv_diag), colour, tb);
      else
        launch_pdl(k_gs_fast<DISC, VARNU, GRP, T, LP, 1>, gg.grd, gg.blk, s, g, u + cs, rhs + cs, T(inv_diag),
                   colour, tb);
    }
  });
}
#endif

#if (!defined(HHG_FAST_ONLY) || HHG_FAST_ONLY == 64) && !defined(HHG_FAST_BATCHED)
int fast_terms(int disc, int varnu, int op) {
#define HHG_N(D, V, O) if (disc == D && varnu == V && op == O) return gen::S<D, V, O>::N;
  HHG_N(1, 0, OP_FULL) HHG_N(1, 0, OP_A) HHG_N(1, 0, OP_BT) HHG_N(1, 0, OP_BC)
  HHG_N(1, 1, OP_FULL) HHG_N(1, 1, OP_A) HHG_N(1, 1, OP_BT) HHG_N(1, 1, OP_BC)
  HHG_N(2, 0, OP_FULL) HHG_N(2, 0, OP_A) HHG_N(2, 0, OP_BT) HHG_N(2, 0, OP_BC)
  HHG_N(2, 1, OP_FULL) HHG_N(2, 1, OP_A) HHG_N(2, 1, OP_BT) HHG_N(2, 1, OP_BC)
#undef HHG_N
  return -1;
}

#endif

#if defined(HHG_FAST_BATCHED)
// run-time dispatch over (disc, varnu, op) of the recorders
template <class T>
void fast_rows_record(int disc, int varnu, int op, const Geo& g, const OpDev& od, const void* tab, int mode,
                      const T* x, const T* b, T* y, double alpha, const Shape& sh) {
#define HHG_R(D, V, O) \
  if (disc == D && varnu == V && op == O) return record_rows<D, V, O, T>(g, od, tab, mode, x, b, y, alpha, sh);
  HHG_R(1, 0, OP_FULL) HHG_R(1, 0, OP_BT) HHG_R(1, 0, OP_BC)
  HHG_R(1, 1, OP_FULL) HHG_R(1, 1, OP_BT) HHG_R(1, 1, OP_BC)
  HHG_R(2, 0, OP_FULL) HHG_R(2, 0, OP_BT) HHG_R(2, 0, OP_BC)
  HHG_R(2, 1, OP_FULL) HHG_R(2, 1, OP_BT) HHG_R(2, 1, OP_BC)
#undef HHG_R
}

template <class T>
void fast_gs_record(int disc, int varnu, const Geo& g, const void* tab, int grp, int colour, double inv_diag, T* u,
                    const T* rhs, const Shape& sh, int comp) {
  if (disc == 1 && !varnu) record_gs<1, 0, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp);
  else if (disc == 1) record_gs<1, 1, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp);
  else if (!varnu) record_gs<2, 0, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp);
  else record_gs<2, 1, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp);
}

#if HHG_FAST_ONLY == 64
template void fast_rows_record<double>(int, int, int, const Geo&, const OpDev&, const void*, int, const double*,
                                       const double*, double*, double, const Shape&);
template void fast_gs_record<double>(int, int, const Geo&, const void*, int, int, double, double*, const double*,
                                     const Shape&, int);
#else
template void fast_rows_record<float>(int, int, int, const Geo&, const OpDev&, const void*, int, const float*,
                                      const float*, float*, double, const Shape&);
template void fast_gs_record<float>(int, int, const Geo&, const void*, int, int, double, float*, const float*,
                                    const Shape&, int);
#endif
#else
// run-time dispatch over (disc, varnu, op); while a batch records, the
// recorders (the batched translation units) take the launch
template <class T>
void fast_rows(int disc, int varnu, int op, const Geo& g, const OpDev& od, const void* tab, int mode, const T* x,
               const T* b, T* y, double alpha, const Shape& sh, cudaStream_t s) {
  if (g_rec) return fast_rows_record<T>(disc, varnu, op, g, od, tab, mode, x, b, y, alpha, sh);
#define HHG_R(D, V, O) \
  if (disc == D && varnu == V && op == O) return launch_rows_fast<D, V, O, T>(g, od, tab, mode, x, b, y, alpha, sh, s);
  HHG_R(1, 0, OP_FULL) HHG_R(1, 0, OP_BT) HHG_R(1, 0, OP_BC)
  HHG_R(1, 1, OP_FULL) HHG_R(1, 1, OP_BT) HHG_R(1, 1, OP_BC)
  HHG_R(2, 0, OP_FULL) HHG_R(2, 0, OP_BT) HHG_R(2, 0, OP_BC)
  HHG_R(2, 1, OP_FULL) HHG_R(2, 1, OP_BT) HHG_R(2, 1, OP_BC)
#undef HHG_R
}

template <class T>
void fast_gs(int disc, int varnu, const Geo& g, const void* tab, int grp, int colour, double inv_diag, T* u,
             const T* rhs, const Shape& sh, cudaStream_t s, int comp) {
  if (g_rec) return fast_gs_record<T>(disc, varnu, g, tab, grp, colour, inv_diag, u, rhs, sh, comp);
  if (disc == 1 && !varnu) launch_gs_fast<1, 0, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp, s);
  else if (disc == 1) launch_gs_fast<1, 1, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp, s);
  else if (!varnu) launch_gs_fast<2, 0, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp, s);
  else launch_gs_fast<2, 1, T>(g, tab, grp, colour, inv_diag, u, rhs, sh, comp, s);
}

// HHG_FAST_ONLY = 64 / 32 compiles one precision (the build compiles this
// file once per precision, in parallel)
#if !defined(HHG_FAST_ONLY) || HHG_FAST_ONLY == 64
template void fast_rows<double>(int, int, int, const Geo&, const OpDev&, const void*, int, const double*, const double*,
                                double*, double, const Shape&, cudaStream_t);
template void fast_gs<double>(int, int, const Geo&, const void*, int, int, double, double*, const double*, const Shape&,
                              cudaStream_t, int);
#endif
#if !defined(HHG_FAST_ONLY) || HHG_FAST_ONLY == 32
template void fast_rows<float>(int, int, int, const Geo&, const OpDev&, const void*, int, const float*, const float*,
                               float*, double, const Shape&, cudaStream_t);
template void fast_gs<float>(int, int, const Geo&, const void*, int, int, double, float*, const float*, const Shape&,
                             cudaStream_t, int);
#endif
#endif

}  // namespace hhg
