// Cluster-resident inexact Uzawa smoother for the small levels of the
// hierarchy (Sec. 3.2, Eqs. uzawa-velocity / uzawa-pressure).
//
// On the coarse levels of a V-cycle every phase of the smoother (the B^T
// residual, each Gauss-Seidel colour or edge group, the (B, -C) residual and
// the pressure update) touches only a few thousand DoFs, so one kernel launch
// per phase costs more than the phase itself.  Here one launch of a single
// thread-block cluster (1..8 CTAs of 1024 threads) runs all phases of all
// requested Uzawa iterations, with a cluster barrier (release / acquire)
// between phases.  Values written inside the kernel are read with L2-coherent
// loads (ld.global.cg), never through the non-coherent read-only path.
// Phase order, arithmetic and the row/term order are those of fast.cu, so the
// result equals the per-phase launches up to the order of independent updates
// (which do not interact).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "fast.h"
#include "kernels.h"
#include "small.h"
#include "structure.inc"

namespace cg = cooperative_groups;

namespace hhg {
namespace {

template <class T> __device__ __forceinline__ T ldc(const T* p) { return __ldcg(p); }

__device__ __forceinline__ int64_t ssite(const Geo& g, int i, int j, int k) {
  return int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy;
}

template <class S, int R, class F>
__device__ __forceinline__ void sdispatch(int r, F&& f) {
  if constexpr (R < S::R) {
    if (r == R) f(std::integral_constant<int, R>{});
    else sdispatch<S, R + 1>(r, f);
  }
}

template <int T0, int N, class T, class Tab>
__device__ __forceinline__ T sseg(const Tab& tab, const T* xs) {
  T a = T(0);
#pragma unroll
  for (int t = 0; t < N; ++t) a += tab.w[T0 + t] * ldc(xs + tab.off[T0 + t]);
  return a;
}

template <class T> __device__ __forceinline__ T sbw(const OpDev& op, int t);
template <> __device__ __forceinline__ double sbw<double>(const OpDev& op, int t) { return op.bw64[t]; }
template <> __device__ __forceinline__ float sbw<float>(const OpDev& op, int t) { return op.bw32[t]; }

// y = b - (row of S at site (i,j,k)), boundary rules as in fast.cu
template <int VARNU, int OUT, int OG, int ALL, int T0, int N0, int N1, int N2, class T, class Tab>
__device__ __forceinline__ void sres_row(const Geo& g, int R, int i, int j, int k, const T* x, const T* b, T* y,
                                         const OpDev& op, const Tab& tab) {
  constexpr int ox = OG == 1 || OG == 4 || OG == 5 || OG == 7;
  constexpr int oy = OG == 2 || OG == 4 || OG == 6 || OG == 7;
  constexpr int oz = OG == 3 || OG == 5 || OG == 6 || OG == 7;
  if (i > g.nx - ox || j > g.ny - oy || k > g.nz - oz) return;
  const int64_t idx = ssite(g, i, j, k);
  const int Px = 2 * i + ox, Py = 2 * j + oy, Pz = 2 * k + oz;
  const bool bnd = Px == 0 || Py == 0 || Pz == 0 || Px == 2 * g.nx || Py == 2 * g.ny || Pz == 2 * g.nz;
  T* yo = y + int64_t(OUT) * g.arr + idx;
  if (bnd && !ALL) {
    *yo = T(0);
    return;
  }
  const T* xs = x + idx;
  const T a0 = sseg<T0, N0, T>(tab, xs);
  const T a1 = sseg<T0 + N0, N1, T>(tab, xs);
  T a2;
  if (!bnd) {
    a2 = sseg<T0 + N0 + N1, N2, T>(tab, xs);
  } else {
    a2 = T(0);
    if (N2 > 0) {
      const DRow row = op.rows[R];
      for (int t = row.b0 + row.m0 + row.m1; t < row.b0 + row.m0 + row.m1 + row.m2; ++t) {
        const DTermB tm = op.bterms[t];
        const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
        if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
        a2 += sbw<T>(op, t) * ldc(x + int64_t(tm.arr) * g.arr + idx + tm.off);
      }
    }
  }
  T v = a0;
  if (VARNU) {
    v += T(g.esc[k]) * a1 + T(g.eisc[k]) * a2;
  } else {
    v += a1 + a2;
  }
  *yo = ldc(b + int64_t(OUT) * g.arr + idx) - v;
}

template <int VARNU, int GRP, int T0, int N1, class T, class Tab>
__device__ __forceinline__ void sgs(const Geo& g, int i, int j, int k, T* u, const T* rhs, T inv_diag,
                                    const Tab& tab) {
  constexpr int ox = GRP == 1 || GRP == 4 || GRP == 5 || GRP == 7;
  constexpr int oy = GRP == 2 || GRP == 4 || GRP == 6 || GRP == 7;
  constexpr int oz = GRP == 3 || GRP == 5 || GRP == 6 || GRP == 7;
  const int Px = 2 * i + ox, Py = 2 * j + oy, Pz = 2 * k + oz;
  if (Px <= 0 || Py <= 0 || Pz <= 0 || Px >= 2 * g.nx || Py >= 2 * g.ny || Pz >= 2 * g.nz) return;
  const int64_t idx = ssite(g, i, j, k);
  const int64_t cs = int64_t(g.G) * g.arr;
  const T* us = u + idx;
  T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
  for (int t = 1; t < N1; ++t) {
    const T wt = tab.w[T0 + t];
    const int o = tab.off[T0 + t];
    a0 += wt * ldc(us + o);
    a1 += wt * ldc(us + o + cs);
    a2 += wt * ldc(us + o + 2 * cs);
  }
  T einv = T(1);
  if (VARNU) einv = T(g.eisc[k]);
  const int64_t o0 = int64_t(GRP) * g.arr + idx;
  u[o0] = (ldc(rhs + o0) * einv - a0) * inv_diag;
  u[o0 + cs] = (ldc(rhs + o0 + cs) * einv - a1) * inv_diag;
  u[o0 + 2 * cs] = (ldc(rhs + o0 + 2 * cs) * einv - a2) * inv_diag;
}

template <int DISC, int VARNU, class T>
__global__ void __launch_bounds__(1024)
    k_uzawa_cluster(Geo g, T* x, const T* b, T* tmp, const double* inv_ml, SmallArgs a, OpDev bc_op,
                    const __grid_constant__ SmallTabs<DISC, VARNU, T> tabs) {
  using SA = gen::S<DISC, VARNU, OP_A>;
  using SBT = gen::S<DISC, VARNU, OP_BT>;
  using SBC = gen::S<DISC, VARNU, OP_BC>;
  cg::cluster_group cluster = cg::this_cluster();
  const int nthr = int(gridDim.x * blockDim.x);
  const int tid = int(blockIdx.x * blockDim.x + threadIdx.x);
  const int nxp = g.nx + 1, nyp = g.ny + 1, nzp = g.nz + 1;
  const int V = nxp * nyp * nzp;
  const int64_t po = 3 * int64_t(g.G) * g.arr;
  constexpr int G = DISC == 1 ? 1 : 8;
  for (int it = 0; it < a.iterations; ++it) {
    // velocity step: tmp_u = b_u - B^T p
    for (int q = tid; q < SBT::R * V; q += nthr) {
      const int r = q / V, s = q - r * V;
      const int k = s / (nxp * nyp), rem = s - k * nxp * nyp, j = rem / nxp, i = rem - j * nxp;
      sdispatch<SBT, 0>(r, [&](auto rc) {
        constexpr int R = decltype(rc)::value;
        constexpr gen::RowS rw = SBT::rows[R];
        sres_row<VARNU, rw.out, rw.og, rw.all, rw.t0, rw.n0, rw.n1, rw.n2>(g, R, i, j, k, x, b, tmp, bc_op, tabs.BT);
      });
    }
    cluster.sync();
    // xi Gauss-Seidel sweeps on A u = tmp_u (forward, and backward for A_s)
    const int nph = 4 + (G - 1);
    for (int sw = 0; sw < a.xi; ++sw) {
      for (int pass = 0; pass < (a.ahat == HHG_AHAT_S ? 2 : 1); ++pass) {
        for (int pi = 0; pi < nph; ++pi) {
          const int ph = pass == 0 ? pi : nph - 1 - pi;
          const int grp = ph < 4 ? 0 : ph - 3;
          const int colour = ph < 4 ? ph : -1;
          const int w = colour >= 0 ? (nxp + 3) / 4 : nxp;
          for (int q = tid; q < w * nyp * nzp; q += nthr) {
            const int k = q / (w * nyp), rem = q - k * w * nyp, j = rem / w;
            int i = rem - j * w;
            if (colour >= 0) i = 4 * i + (((colour - j - k) % 4) + 4) % 4;
            sdispatch<SA, 0>(grp, [&](auto rc) {
              constexpr int GR = decltype(rc)::value;
              if constexpr (GR < G) {
                constexpr gen::RowS rw = SA::rows[GR];
                sgs<VARNU, GR, rw.t0, rw.n1>(g, i, j, k, x, tmp, T(a.inv_diag[GR]), tabs.A);
              }
            });
          }
          cluster.sync();
        }
      }
    }
    // pressure step: tmp_p = g - (B u - C p), then p -= tmp_p / (omega^{-1} M_L)
    for (int q = tid; q < V; q += nthr) {
      const int k = q / (nxp * nyp), rem = q - k * nxp * nyp, j = rem / nxp, i = rem - j * nxp;
      constexpr gen::RowS rw = SBC::rows[0];
      sres_row<VARNU, rw.out, rw.og, rw.all, rw.t0, rw.n0, rw.n1, rw.n2>(g, 0, i, j, k, x, b, tmp, bc_op, tabs.BC);
    }
    cluster.sync();
    for (int q = tid; q < V; q += nthr) {
      const int k = q / (nxp * nyp), rem = q - k * nxp * nyp, j = rem / nxp, i = rem - j * nxp;
      const int64_t idx = ssite(g, i, j, k);
      x[po + idx] -= T(a.inv_omega_inv * inv_ml[idx]) * ldc(tmp + po + idx);
    }
    cluster.sync();
  }
}

}  // namespace

template <int DISC, int VARNU, class T>
int launch_uzawa_cluster(const Geo& g, T* x, const T* b, T* tmp, const double* inv_ml, const SmallArgs& a,
                         const OpDev& bc_op, const void* tabs, cudaStream_t s) {
  using Tabs = SmallTabs<DISC, VARNU, T>;
  const int64_t V = int64_t(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
  int cl = int((V * 3 + 4095) / 4096);            // CTAs: about 4 DoF sites per thread
  if (cl < 1) cl = 1;
  if (cl > 8) cl = 8;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cl, 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  ++g_launches;
  const Tabs& tb = *static_cast<const Tabs*>(tabs);
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_uzawa_cluster<DISC, VARNU, T>, g, x, b, tmp, inv_ml, a, bc_op, tb);
  return e == cudaSuccess ? 0 : -1;
}

template <class T>
int uzawa_cluster(int disc, int varnu, const Geo& g, T* x, const T* b, T* tmp, const double* inv_ml,
                  const SmallArgs& a, const OpDev& bc_op, const void* tabs, cudaStream_t s) {
  if (disc == 1 && !varnu) return launch_uzawa_cluster<1, 0, T>(g, x, b, tmp, inv_ml, a, bc_op, tabs, s);
  if (disc == 1) return launch_uzawa_cluster<1, 1, T>(g, x, b, tmp, inv_ml, a, bc_op, tabs, s);
  if (!varnu) return launch_uzawa_cluster<2, 0, T>(g, x, b, tmp, inv_ml, a, bc_op, tabs, s);
  return launch_uzawa_cluster<2, 1, T>(g, x, b, tmp, inv_ml, a, bc_op, tabs, s);
}

size_t small_tabs_bytes(int disc, int varnu, int prec) {
  if (prec == HHG_FP64) {
    if (disc == 1) return varnu ? sizeof(SmallTabs<1, 1, double>) : sizeof(SmallTabs<1, 0, double>);
    return varnu ? sizeof(SmallTabs<2, 1, double>) : sizeof(SmallTabs<2, 0, double>);
  }
  if (disc == 1) return varnu ? sizeof(SmallTabs<1, 1, float>) : sizeof(SmallTabs<1, 0, float>);
  return varnu ? sizeof(SmallTabs<2, 1, float>) : sizeof(SmallTabs<2, 0, float>);
}

size_t small_tabs_offset(int disc, int varnu, int prec, int which) {
#define HHG_OFFS(D, V, T)                                                  \
  if (disc == D && varnu == V) {                                           \
    using ST = SmallTabs<D, V, T>;                                         \
    return which == 0 ? offsetof(ST, A) : which == 1 ? offsetof(ST, BT) : offsetof(ST, BC); \
  }
  if (prec == HHG_FP64) {
    HHG_OFFS(1, 0, double) HHG_OFFS(1, 1, double) HHG_OFFS(2, 0, double) HHG_OFFS(2, 1, double)
  } else {
    HHG_OFFS(1, 0, float) HHG_OFFS(1, 1, float) HHG_OFFS(2, 0, float) HHG_OFFS(2, 1, float)
  }
#undef HHG_OFFS
  return 0;
}

template int uzawa_cluster<double>(int, int, const Geo&, double*, const double*, double*, const double*,
                                   const SmallArgs&, const OpDev&, const void*, cudaStream_t);
template int uzawa_cluster<float>(int, int, const Geo&, float*, const float*, float*, const double*,
                                  const SmallArgs&, const OpDev&, const void*, cudaStream_t);

}  // namespace hhg
