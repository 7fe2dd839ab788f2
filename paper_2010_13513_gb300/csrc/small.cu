// Shared-memory-resident inexact Uzawa smoother for the small levels of the
// hierarchy (Sec. 3.2, Eqs. uzawa-velocity / uzawa-pressure).
//
// On the coarse levels of a V-cycle every phase of the smoother (the B^T
// residual, each Gauss-Seidel colour or edge group, the (B, -C) residual and
// the pressure update) touches only a few thousand DoFs, so one kernel launch
// per phase, with every stencil term a round trip to L2, costs far more than
// the arithmetic.  Here one launch of a thread-block cluster of C CTAs
// (1 <= C <= 16) runs all phases of all requested Uzawa iterations with the
// level's block vector held in shared memory:
//
//  * CTA c owns the k planes [c (nz+1) / C, (c+1) (nz+1) / C) of every array
//    (velocity groups and pressure) and stores them, plus one halo plane
//    below and above, in the global array layout with a local array stride,
//    so the stencil offsets keep their in-array part (di + dj sx + dk sy);
//  * a phase updates the CTA's own sites from shared memory; after a cluster
//    barrier every CTA copies the sites the phase changed in its neighbours'
//    boundary planes into its own halo planes (distributed shared memory);
//  * the right-hand side is read through the read-only path; the residuals
//    tmp = b - B^T p and g - (B u - C p) go to global memory and are read back
//    only by the CTA that wrote them (visible after __syncthreads).
//
// A phase only ever updates sites that no site of the same phase reads (a
// vertex colour, or one edge group), so the copy after phase p never races
// with the writes of phase p+1.  The one exception, the same phase twice in a
// row at the turn of a symmetric sweep, is skipped: with no coupling inside a
// phase its second application reproduces the same values.  Phase order,
// arithmetic and the row/term order are those of fast.cu, so the iterates
// equal those of the per-phase launches.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <type_traits>

#include "fast.h"
#include "kernels.h"
#include "small.h"
#include "structure.inc"

namespace cg = cooperative_groups;

namespace hhg {
namespace {

template <class S, int R, class F>
__device__ __forceinline__ void sdispatch(int r, F&& f) {
  if constexpr (R < S::R) {
    if (r == R) f(std::integral_constant<int, R>{});
    else sdispatch<S, R + 1>(r, f);
  }
}

template <int T0, int N, class T, class Tab>
__device__ __forceinline__ T sseg(const Tab& tab, const T* xl) {
  T a = T(0);
#pragma unroll
  for (int t = 0; t < N; ++t) a += tab.w[T0 + t] * xl[tab.off[T0 + t]];
  return a;
}

template <class T> __device__ __forceinline__ T sbw(const OpDev& op, int t);
template <> __device__ __forceinline__ double sbw<double>(const OpDev& op, int t) { return __ldg(op.bw64 + t); }
template <> __device__ __forceinline__ float sbw<float>(const OpDev& op, int t) { return __ldg(op.bw32 + t); }

// y = b - (row of S at site (i,j,k)); x from the shared slab (local index il,
// local array stride arr_l), b and y in global memory (index ig); boundary
// rules as in fast.cu
template <int VARNU, int OUT, int OG, int ALL, int T0, int N0, int N1, int N2, class T, class Tab>
__device__ __forceinline__ void rres_row(const Geo& g, int arr_l, int R, int i, int j, int k, int64_t ig, int il,
                                         const T* xs, const T* __restrict__ b, T* y, const OpDev& op,
                                         const Tab& tab) {
  constexpr int ox = OG == 1 || OG == 4 || OG == 5 || OG == 7;
  constexpr int oy = OG == 2 || OG == 4 || OG == 6 || OG == 7;
  constexpr int oz = OG == 3 || OG == 5 || OG == 6 || OG == 7;
  if (i > g.nx - ox || j > g.ny - oy || k > g.nz - oz) return;
  const int Px = 2 * i + ox, Py = 2 * j + oy, Pz = 2 * k + oz;
  const bool bnd = Px == 0 || Py == 0 || Pz == 0 || Px == 2 * g.nx || Py == 2 * g.ny || Pz == 2 * g.nz;
  T* yo = y + int64_t(OUT) * g.arr + ig;
  if (bnd && !ALL) {
    *yo = T(0);
    return;
  }
  const T* xl = xs + il;
  const T a0 = sseg<T0, N0, T>(tab, xl);
  const T a1 = sseg<T0 + N0, N1, T>(tab, xl);
  T a2;
  if (!bnd) {
    a2 = sseg<T0 + N0 + N1, N2, T>(tab, xl);
  } else {
    a2 = T(0);
    if (N2 > 0) {
      const DRow row = op.rows[R];
      for (int t = row.b0 + row.m0 + row.m1; t < row.b0 + row.m0 + row.m1 + row.m2; ++t) {
        const DTermB tm = op.bterms[t];
        const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
        if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
        a2 += sbw<T>(op, t) * xs[tm.arr * arr_l + il + tm.off];
      }
    }
  }
  T v = a0;
  if (VARNU) {
    v += T(g.esc[k]) * a1 + T(g.eisc[k]) * a2;
  } else {
    v += a1 + a2;
  }
  *yo = __ldg(b + int64_t(OUT) * g.arr + ig) - v;
}

// one Gauss-Seidel update of the three velocity components of group GRP at
// site (i,j,k) (Dirichlet sites are left alone)
template <int VARNU, int GRP, int T0, int N1, class T, class Tab>
__device__ __forceinline__ void rgs(const Geo& g, int arr_l, int i, int j, int k, int64_t ig, int il, T* xs,
                                    const T* tmp, T inv_diag, const Tab& tab) {
  constexpr int ox = GRP == 1 || GRP == 4 || GRP == 5 || GRP == 7;
  constexpr int oy = GRP == 2 || GRP == 4 || GRP == 6 || GRP == 7;
  constexpr int oz = GRP == 3 || GRP == 5 || GRP == 6 || GRP == 7;
  const int Px = 2 * i + ox, Py = 2 * j + oy, Pz = 2 * k + oz;
  if (Px <= 0 || Py <= 0 || Pz <= 0 || Px >= 2 * g.nx || Py >= 2 * g.ny || Pz >= 2 * g.nz) return;
  const int csl = g.G * arr_l;
  const T* us = xs + il;
  T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll
  for (int t = 1; t < N1; ++t) {               // the diagonal is the first term
    const T wt = tab.w[T0 + t];
    const int o = tab.off[T0 + t];
    a0 += wt * us[o];
    a1 += wt * us[o + csl];
    a2 += wt * us[o + 2 * csl];
  }
  T einv = T(1);
  if (VARNU) einv = T(g.eisc[k]);
  const int ol = GRP * arr_l + il;
  const int64_t og = int64_t(GRP) * g.arr + ig, csg = int64_t(g.G) * g.arr;
  xs[ol] = (tmp[og] * einv - a0) * inv_diag;
  xs[ol + csl] = (tmp[og + csg] * einv - a1) * inv_diag;
  xs[ol + 2 * csl] = (tmp[og + 2 * csg] * einv - a2) * inv_diag;
}

template <int DISC, int VARNU, class T>
__global__ void __launch_bounds__(kResidentThreads)
    k_uzawa_resident(Geo g, int arr_l, T* xg, const T* __restrict__ b, T* tmp, const double* __restrict__ inv_ml,
                     SmallArgs a, OpDev bc_op, const __grid_constant__ SmallTabs<DISC, VARNU, T> tabs) {
  using SA = gen::S<DISC, VARNU, OP_A>;
  using SBT = gen::S<DISC, VARNU, OP_BT>;
  using SBC = gen::S<DISC, VARNU, OP_BC>;
  constexpr int G = DISC == 1 ? 1 : 8;
  constexpr int NA = 3 * G + 1;                 // arrays of the block vector
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);
  cg::cluster_group cluster = cg::this_cluster();
  const int C = int(cluster.num_blocks()), c = int(cluster.block_rank());
  const int nxp = g.nx + 1, nyp = g.ny + 1, nzp = g.nz + 1;
  const int kb = c * nzp / C, ke = (c + 1) * nzp / C, nk = ke - kb;
  const int sx = g.sx, sy = int(g.sy);
  const int tid = int(threadIdx.x), nthr = int(blockDim.x);
  auto bar = [&] {
    if (C > 1) cluster.sync();
    else __syncthreads();
  };
  // owned planes kb .. ke-1 and the halo planes kb-1, ke (global plane k
  // starts at (k+1) sy, local plane k-kb+1 at (k-kb+1) sy)
  {
    const int span = (nk + 2) * sy;
    for (int q = tid; q < NA * span; q += nthr) {
      const int ar = q / span, r = q - ar * span;
      xs[ar * arr_l + r] = xg[int64_t(ar) * g.arr + int64_t(kb) * sy + r];
    }
  }
  bar();                                         // every CTA of the cluster runs before any remote access

  // copy the sites of arrays a0, a0+astep, ... (na arrays) that the last
  // phase changed from the neighbours' boundary planes into the halo planes
  auto pull = [&](int a0, int na, int astep, int colour) {
    if (C == 1) return;
    for (int side = 0; side < 2; ++side) {
      if ((side == 0 && c == 0) || (side == 1 && c == C - 1)) continue;
      const int nb = side == 0 ? c - 1 : c + 1;
      const int kh = side == 0 ? kb - 1 : ke;          // global plane of the halo
      const int src = kh - nb * nzp / C + 1;           // its local plane in the neighbour
      const int dst = side == 0 ? 0 : nk + 1;
      const T* rem = cluster.map_shared_rank(xs, nb);
      for (int q = tid; q < na * sy; q += nthr) {
        const int aa = q / sy, e = q - aa * sy;
        if (colour >= 0) {
          const int jj = e / sx - 1, ii = e - (jj + 1) * sx - 1;
          if (ii < 0 || jj < 0 || ii > g.nx || jj > g.ny || ((ii + jj + kh) & 3) != colour) continue;
        }
        const int ar = a0 + aa * astep;
        xs[ar * arr_l + dst * sy + e] = rem[ar * arr_l + src * sy + e];
      }
    }
    __syncthreads();
  };

  const int plane = nxp * nyp, Vl = plane * nk;
  const int64_t pog = 3 * int64_t(G) * g.arr;
  const int pol = 3 * G * arr_l;
  for (int it = 0; it < a.iterations; ++it) {
    // velocity step: tmp_u = b_u - B^T p
    for (int q = tid; q < SBT::R * Vl; q += nthr) {
      const int r = q / Vl, s = q - r * Vl;
      const int kl = s / plane, rem = s - kl * plane, j = rem / nxp, i = rem - j * nxp;
      const int k = kb + kl;
      const int il = (i + 1) + (j + 1) * sx + (kl + 1) * sy;
      const int64_t ig = int64_t(i + 1) + int64_t(j + 1) * sx + int64_t(k + 1) * sy;
      sdispatch<SBT, 0>(r, [&](auto rc) {
        constexpr int R = decltype(rc)::value;
        constexpr gen::RowS rw = SBT::rows[R];
        rres_row<VARNU, rw.out, rw.og, rw.all, rw.t0, rw.n0, rw.n1, rw.n2>(g, arr_l, R, i, j, k, ig, il, xs, b, tmp,
                                                                           bc_op, tabs.BT);
      });
    }
    __syncthreads();
    // xi Gauss-Seidel sweeps on A u = tmp_u (forward, and backward for A_s)
    constexpr int nph = 4 + (G - 1);
    int prev = -1;
    for (int sw = 0; sw < a.xi; ++sw) {
      for (int pass = 0; pass < (a.ahat == HHG_AHAT_S ? 2 : 1); ++pass) {
        for (int pi = 0; pi < nph; ++pi) {
          const int ph = pass == 0 ? pi : nph - 1 - pi;
          if (ph == prev) continue;
          prev = ph;
          const int grp = ph < 4 ? 0 : ph - 3;
          const int colour = ph < 4 ? ph : -1;
          const int w = colour >= 0 ? (nxp + 3) / 4 : nxp;
          for (int q = tid; q < w * nyp * nk; q += nthr) {
            const int kl = q / (w * nyp), rem = q - kl * w * nyp, j = rem / w;
            const int k = kb + kl;
            int i = rem - j * w;
            if (colour >= 0) i = 4 * i + (((colour - j - k) % 4) + 4) % 4;
            const int il = (i + 1) + (j + 1) * sx + (kl + 1) * sy;
            const int64_t ig = int64_t(i + 1) + int64_t(j + 1) * sx + int64_t(k + 1) * sy;
            sdispatch<SA, 0>(grp, [&](auto rc) {
              constexpr int GR = decltype(rc)::value;
              if constexpr (GR < G) {
                constexpr gen::RowS rw = SA::rows[GR];
                rgs<VARNU, GR, rw.t0, rw.n1>(g, arr_l, i, j, k, ig, il, xs, tmp, T(a.inv_diag[GR]), tabs.A);
              }
            });
          }
          bar();
          pull(grp, 3, G, colour);
        }
      }
    }
    // pressure step: tmp_p = g - (B u - C p), then p -= tmp_p / (omega^{-1} M_L)
    for (int q = tid; q < Vl; q += nthr) {
      const int kl = q / plane, rem = q - kl * plane, j = rem / nxp, i = rem - j * nxp;
      const int k = kb + kl;
      const int il = (i + 1) + (j + 1) * sx + (kl + 1) * sy;
      const int64_t ig = int64_t(i + 1) + int64_t(j + 1) * sx + int64_t(k + 1) * sy;
      constexpr gen::RowS rw = SBC::rows[0];
      rres_row<VARNU, rw.out, rw.og, rw.all, rw.t0, rw.n0, rw.n1, rw.n2>(g, arr_l, 0, i, j, k, ig, il, xs, b, tmp,
                                                                         bc_op, tabs.BC);
    }
    __syncthreads();
    for (int q = tid; q < Vl; q += nthr) {
      const int kl = q / plane, rem = q - kl * plane, j = rem / nxp, i = rem - j * nxp;
      const int il = (i + 1) + (j + 1) * sx + (kl + 1) * sy;
      const int64_t ig = int64_t(i + 1) + int64_t(j + 1) * sx + int64_t(kb + kl + 1) * sy;
      xs[pol + il] -= T(a.inv_omega_inv * inv_ml[ig]) * tmp[pog + ig];
    }
    bar();
    pull(3 * G, 1, 1, -1);
  }
  // owned planes back to global memory
  {
    const int span = nk * sy;
    for (int q = tid; q < NA * span; q += nthr) {
      const int ar = q / span, r = q - ar * span;
      xg[int64_t(ar) * g.arr + int64_t(kb + 1) * sy + r] = xs[ar * arr_l + sy + r];
    }
  }
  if (C > 1) cluster.sync();                     // no CTA leaves while a neighbour may read its shared memory
}

template <class T> constexpr int prec_of() { return sizeof(T) == 8 ? HHG_FP64 : HHG_FP32; }

void fill_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int C, size_t smem, cudaStream_t s) {
  cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(kResidentThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

template <int DISC, int VARNU, class T>
bool feasible_impl(const Geo& g, int C) {
  if (C < 1 || C > kResidentMaxCtas || C > g.nz + 1) return false;
  const size_t smem = resident_smem(g, C, prec_of<T>());
  if (smem > kResidentSmemMax) return false;
  auto fn = k_uzawa_resident<DISC, VARNU, T>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kResidentSmemMax)) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, C, smem, nullptr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

template <int DISC, int VARNU, class T>
int launch_resident(const Geo& g, int C, T* x, const T* b, T* tmp, const double* inv_ml, const SmallArgs& a,
                    const OpDev& bc_op, const void* tabs, cudaStream_t s) {
  using Tabs = SmallTabs<DISC, VARNU, T>;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, C, resident_smem(g, C, prec_of<T>()), s);
  ++g_launches;
  const Tabs& tb = *static_cast<const Tabs*>(tabs);
  const int arr_l = int(resident_arr(g, C));
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_uzawa_resident<DISC, VARNU, T>, g, arr_l, x, b, tmp, inv_ml, a, bc_op, tb);
  return e == cudaSuccess ? 0 : -1;
}

template <class T, int N>
bool localise_tab(FastTab<T, N>& tab, const Geo& g, int64_t arr_l) {
  const int64_t na = 3 * int64_t(g.G) + 1;
  for (int t = 0; t < N; ++t) {
    const int64_t off = tab.off[t];
    const int64_t ar = std::llround(double(off) / double(g.arr));
    const int64_t rel = off - ar * g.arr;
    const int64_t dk = std::llround(double(rel) / double(g.sy));
    const int64_t dj = std::llround(double(rel - dk * g.sy) / double(g.sx));
    const int64_t di = rel - dk * g.sy - dj * g.sx;
    if (ar < 0 || ar >= na || dk < -1 || dk > 1 || dj < -1 || dj > 1 || di < -1 || di > 1) return false;
    tab.off[t] = int(ar * arr_l + rel);
  }
  return true;
}

template <int D, int V, class T>
bool localise_impl(const std::vector<char>& in, const Geo& g, int64_t arr_l, std::vector<char>& out) {
  using ST = SmallTabs<D, V, T>;
  if (in.size() != sizeof(ST)) return false;
  out = in;
  ST* st = reinterpret_cast<ST*>(out.data());
  return localise_tab(st->A, g, arr_l) && localise_tab(st->BT, g, arr_l) && localise_tab(st->BC, g, arr_l);
}

}  // namespace

int64_t resident_arr(const Geo& g, int ctas) {
  const int64_t nzp = g.nz + 1;
  const int64_t planes = (nzp + ctas - 1) / ctas + 2;
  return (planes * g.sy + 3) / 4 * 4;
}

size_t resident_smem(const Geo& g, int ctas, int prec) {
  const size_t es = prec == HHG_FP64 ? 8 : 4;
  return size_t(3 * g.G + 1) * size_t(resident_arr(g, ctas)) * es;
}

bool resident_feasible(int disc, int varnu, int prec, const Geo& g, int ctas) {
  if (prec == HHG_FP64) {
    if (disc == 1) return varnu ? feasible_impl<1, 1, double>(g, ctas) : feasible_impl<1, 0, double>(g, ctas);
    return varnu ? feasible_impl<2, 1, double>(g, ctas) : feasible_impl<2, 0, double>(g, ctas);
  }
  if (disc == 1) return varnu ? feasible_impl<1, 1, float>(g, ctas) : feasible_impl<1, 0, float>(g, ctas);
  return varnu ? feasible_impl<2, 1, float>(g, ctas) : feasible_impl<2, 0, float>(g, ctas);
}

bool small_tabs_localise(int disc, int varnu, int prec, const std::vector<char>& in, const Geo& g, int64_t arr_l,
                         std::vector<char>& out) {
  if (prec == HHG_FP64) {
    if (disc == 1)
      return varnu ? localise_impl<1, 1, double>(in, g, arr_l, out) : localise_impl<1, 0, double>(in, g, arr_l, out);
    return varnu ? localise_impl<2, 1, double>(in, g, arr_l, out) : localise_impl<2, 0, double>(in, g, arr_l, out);
  }
  if (disc == 1)
    return varnu ? localise_impl<1, 1, float>(in, g, arr_l, out) : localise_impl<1, 0, float>(in, g, arr_l, out);
  return varnu ? localise_impl<2, 1, float>(in, g, arr_l, out) : localise_impl<2, 0, float>(in, g, arr_l, out);
}

template <class T>
int uzawa_resident(int disc, int varnu, const Geo& g, int ctas, T* x, const T* b, T* tmp, const double* inv_ml,
                   const SmallArgs& a, const OpDev& bc_op, const void* tabs, cudaStream_t s) {
  if (disc == 1 && !varnu) return launch_resident<1, 0, T>(g, ctas, x, b, tmp, inv_ml, a, bc_op, tabs, s);
  if (disc == 1) return launch_resident<1, 1, T>(g, ctas, x, b, tmp, inv_ml, a, bc_op, tabs, s);
  if (!varnu) return launch_resident<2, 0, T>(g, ctas, x, b, tmp, inv_ml, a, bc_op, tabs, s);
  return launch_resident<2, 1, T>(g, ctas, x, b, tmp, inv_ml, a, bc_op, tabs, s);
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

template int uzawa_resident<double>(int, int, const Geo&, int, double*, const double*, double*, const double*,
                                    const SmallArgs&, const OpDev&, const void*, cudaStream_t);
template int uzawa_resident<float>(int, int, const Geo&, int, float*, const float*, float*, const double*,
                                   const SmallArgs&, const OpDev&, const void*, cudaStream_t);

}  // namespace hhg
