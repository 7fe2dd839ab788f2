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
//    so a stencil offset is array * arr_l + di + dj sx + dk sy;
//  * a phase updates the CTA's own sites from shared memory; a value written
//    to a boundary plane is also stored into the neighbour's halo plane
//    (distributed shared memory), and a cluster barrier ends the phase;
//  * a phase has few sites, so each row is shared by P lanes (P = 1..32,
//    chosen per phase from the number of rows): lane p takes the terms
//    p, p+P, ... and the partial sums are added by a butterfly of shuffles;
//  * the residuals tmp = b - B^T p and g - (B u - C p) and the scaled inverse
//    lumped pressure mass omega M_L^{-1} of the owned planes stay in shared
//    memory too; the right-hand side is read through the read-only path,
//    issued before the row sums so that its latency overlaps them.
//
// A Gauss-Seidel phase only ever updates sites that no site of the same phase
// reads (a vertex colour, or one edge group), so the halo stores of a phase
// never touch values read in that phase.  The same phase twice in a row, at
// the turn of a symmetric sweep, is skipped: with no coupling inside a phase
// its second application reproduces the same values.  The pressure update,
// whose halo stores would reach values the (B, -C) residual reads, follows
// that residual after a cluster barrier.  Phase order and arithmetic are
// those of the per-phase kernels; only the order in which the terms of one
// row are added differs (partial sums per lane).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <type_traits>

#include "batch.h"
#include "kernels.h"
#include "small.h"

namespace cg = cooperative_groups;

namespace hhg {
namespace {

template <class T> __device__ __forceinline__ T bw(const OpDev& op, int t);
template <> __device__ __forceinline__ double bw<double>(const OpDev& op, int t) { return __ldg(op.bw64 + t); }
template <> __device__ __forceinline__ float bw<float>(const OpDev& op, int t) { return __ldg(op.bw32 + t); }

// offset bits of an output group: x for groups 1,4,5,7, y for 2,4,6,7, z for 3,5,6,7
__device__ __forceinline__ int gox(int og) { return (0xB2 >> og) & 1; }
__device__ __forceinline__ int goy(int og) { return (0xD4 >> og) & 1; }
__device__ __forceinline__ int goz(int og) { return (0xE8 >> og) & 1; }

// sum over aligned groups of P lanes (every lane of the warp takes part)
template <int P, class T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int m = P >> 1; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// calls f with the lanes-per-row exponent as a compile-time constant
template <class F>
__device__ __forceinline__ void with_lanes(int lp, F&& f) {
  switch (lp) {
    case 0: f(std::integral_constant<int, 0>{}); break;
    case 1: f(std::integral_constant<int, 1>{}); break;
    case 2: f(std::integral_constant<int, 2>{}); break;
    case 3: f(std::integral_constant<int, 3>{}); break;
    case 4: f(std::integral_constant<int, 4>{}); break;
    default: f(std::integral_constant<int, 5>{}); break;
  }
}

// floor(n / d) for 0 <= n, d < 2^16 from m = floor(2^32 / d) + 1: the
// product n m / 2^32 exceeds n / d by less than n / 2^32 < 1 / d, which never
// reaches the next integer (one wide multiply instead of a division)
__device__ __forceinline__ int qdiv(int n, unsigned long long m) {
  return int((unsigned long long)(unsigned)n * m >> 32);
}
__device__ __forceinline__ unsigned long long qmagic(int d) { return (1ull << 32) / unsigned(d) + 1; }

// one phase of the smoother in one CTA: its rows (instances), lanes per row
// (2^lp), lanes in whole warps, and the mixed-radix decomposition of an
// instance index (up to three divisors with their multipliers) into the row
// kind and the site relative to (i0, j0, kf)
struct PhaseDesc {
  int ninst, lp, total;
  int d0, d1, d2;
  unsigned long long m0, m1, m2;
  int kf, i0, j0;
};

// lanes per row: enough to hide the latency of a row sum, few enough that
// the shuffles (about 30 cycles a level) do not outweigh the terms (about
// eight terms per lane, at most `cap` lanes in the phase)
__device__ __forceinline__ int lanes_log2(int n, int terms, int cap) {
  int lp = 0;
  while (lp < 5 && (1 << lp) * 8 < terms && n * (2 << lp) <= cap) ++lp;
  return lp;
}

__device__ __forceinline__ void set_desc(PhaseDesc& d, int ninst, int terms, int cap, int d0, int d1, int d2, int kf,
                                         int i0, int j0) {
  d.ninst = ninst;
  d.lp = lanes_log2(ninst, terms, cap);
  d.total = ((ninst << d.lp) + 31) & ~31;
  d.d0 = max(d0, 1);
  d.d1 = max(d1, 1);
  d.d2 = max(d2, 1);
  d.m0 = qmagic(d.d0);
  d.m1 = qmagic(d.d1);
  d.m2 = qmagic(d.d2);
  d.kf = kf;
  d.i0 = i0;
  d.j0 = j0;
}

// lanes that may share the rows of a Gauss-Seidel phase
constexpr int kPhaseLanes = 256;

// the smoother of one cluster (the kernel below, or one work item of a
// merged launch over several problems' clusters)
template <class T>
__device__ __forceinline__ void uzawa_resident_body(const Geo& g, int arr_l, int arr_t, T* xg,
                                                    const T* __restrict__ b, const double* __restrict__ inv_ml,
                                                    const SmallArgs& a, const OpDev& bc_op, const ResTabs<T>& tb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PhaseDesc sd[13];                     // GS phases 0..nph-1, then B^T, then (B, -C)
  __shared__ T sdiag[8];
  __shared__ ResRow srowA[8];
  const int G = tb.G, NA = 3 * G + 1;
  // shared memory: the slab (NA arrays of stride arr_l, owned planes plus
  // halos), the residuals of the owned planes (NA arrays of stride arr_t,
  // local plane kl at kl sy), omega M_L^{-1} (one array of stride arr_t), tables
  T* xs = reinterpret_cast<T*>(smem_raw);
  T* ts = xs + NA * arr_l;
  T* mls = ts + NA * arr_t;
  T* sw = mls + arr_t;
  int* soff = reinterpret_cast<int*>(sw + tb.nw);
  cg::cluster_group cluster = cg::this_cluster();
  const int C = int(cluster.num_blocks()), c = int(cluster.block_rank());
  const int nxp = g.nx + 1, nyp = g.ny + 1, nzp = g.nz + 1;
  const int kb = c * nzp / C, ke = (c + 1) * nzp / C, nk = ke - kb;
  const int sx = g.sx, sy = int(g.sy);
  const int tid = int(threadIdx.x), nthr = int(blockDim.x), wbase = tid & ~31;
  const bool varnu = tb.varnu != 0;
  const int nph = 4 + (G - 1);
  // neighbours' slabs: my plane kb is the lower neighbour's upper halo plane
  // (local plane nk_lo + 1), my plane ke-1 the upper neighbour's plane 0
  T* lo = (C > 1 && c > 0) ? cluster.map_shared_rank(xs, c - 1) : nullptr;
  T* hi = (C > 1 && c < C - 1) ? cluster.map_shared_rank(xs, c + 1) : nullptr;
  const int nk_lo = c > 0 ? kb - (c - 1) * nzp / C : 0;
  auto bar = [&] {
    if (C > 1) cluster.sync();
    else __syncthreads();
  };
  auto store = [&](int li, int kl, T v) {          // slab value and its halo copies
    xs[li] = v;
    if (kl == 0 && lo) lo[li + nk_lo * sy] = v;
    if (kl == nk - 1 && hi) hi[li - nk * sy] = v;
  };

  for (int t = tid; t < tb.nw; t += nthr) {
    sw[t] = tb.w[t];
    soff[t] = tb.off[t];
  }
  if (tid < G) {
    sdiag[tid] = T(a.inv_diag[tid]);
    srowA[tid] = tb.A[tid];
  }
  if (tid < nph) {
    // Gauss-Seidel phase: interior sites of the group, i in [1-ox, nx-1],
    // j in [1-oy, ny-1], k in [1-oz, nz-1] within the slab; a vertex colour
    // takes every fourth i of a row
    const int ph = tid, grp = ph < 4 ? 0 : ph - 3, colour = ph < 4 ? ph : -1;
    const int i0 = 1 - gox(grp), j0 = 1 - goy(grp), kf = max(kb, 1 - goz(grp));
    const int nkk = max(0, min(ke, g.nz) - kf), nj = g.ny - j0, nis = colour >= 0 ? (g.nx + 2) / 4 : g.nx - i0;
    set_desc(sd[ph], nis * nj * nkk, tb.A[grp].n1 - 1, kPhaseLanes, nis * nj, nis, 1, kf, i0, j0);
  } else if (tid == nph) {
    // B^T rows of every (component, group) at i < nx, j < ny, k < nz
    const int kf = max(kb, 0), nkk = max(0, min(ke, g.nz) - kf), Vb = g.nx * g.ny * nkk;
    int terms = 0;
    for (int r = 0; r < tb.nbt; ++r) terms = max(terms, tb.BT[r].n0 + tb.BT[r].n1 + tb.BT[r].n2);
    set_desc(sd[nph], tb.nbt * Vb, terms, nthr, Vb, g.nx * g.ny, g.nx, kf, 0, 0);
  } else if (tid == nph + 1) {
    // the pressure row at every pressure site of the owned planes
    set_desc(sd[nph + 1], nxp * nyp * nk, tb.BC.n0 + tb.BC.n1 + tb.BC.n2, nthr, nxp * nyp, nxp, 1, kb, 0, 0);
  }
  // owned planes kb .. ke-1 and the halo planes kb-1, ke (global plane k
  // starts at (k+1) sy, local plane k-kb+1 at (k-kb+1) sy); residuals start
  // at 0 so that the lattice's zero ring stays 0 in the pressure update
  {
    const int span = (nk + 2) * sy;
    for (int q = tid; q < NA * span; q += nthr) {
      const int ar = q / span, r = q - ar * span;
      xs[ar * arr_l + r] = xg[int64_t(ar) * g.arr + int64_t(kb) * sy + r];
    }
    for (int r = tid; r < nk * sy; r += nthr) mls[r] = T(a.inv_omega_inv * inv_ml[int64_t(kb + 1) * sy + r]);
    for (int r = tid; r < NA * arr_t; r += nthr) ts[r] = T(0);
  }
  bar();                                           // every CTA runs before any remote store

  const int pol = 3 * G * arr_l, pot = 3 * G * arr_t;
  const int csl = G * arr_l, cst = G * arr_t;
  const unsigned long long msy = qmagic(sy);
  for (int it = 0; it < a.iterations; ++it) {
    // ---- velocity step: tmp_u = b_u - B^T p at the interior sites of every
    // group (Dirichlet rows are never read)
    if (wbase < sd[nph].total) {
      const PhaseDesc d = sd[nph];
      with_lanes(d.lp, [&](auto lpc) {
        constexpr int LP = decltype(lpc)::value, P = 1 << LP;
        for (int q = tid; q < d.total; q += nthr) {  // whole warps: the shuffles see all lanes
          const int inst = q >> LP, p = q & (P - 1);
          const bool valid = inst < d.ninst;
          int r = 0, i = 0, j = 0, k = d.kf;
          if (valid) {
            r = qdiv(inst, d.m0);
            const int s = inst - r * d.d0, kk = qdiv(s, d.m1), rem = s - kk * d.d1;
            j = qdiv(rem, d.m2);
            i = rem - j * d.d2;
            k += kk;
          }
          const ResRow rw = tb.BT[r];
          const bool ok = valid && (i > 0 || gox(rw.og)) && (j > 0 || goy(rw.og)) && (k > 0 || goz(rw.og));
          const int kl = k - kb;
          const int il = (i + 1) + (j + 1) * sx + (kl + 1) * sy;
          const int64_t ig = int64_t(i + 1) + int64_t(j + 1) * sx + int64_t(k + 1) * sy;
          const T bv = (ok && p == 0) ? __ldg(b + int64_t(rw.out) * g.arr + ig) : T(0);
          T a0 = T(0), a1 = T(0), a2 = T(0);
          if (ok) {
            const T* xl = xs + il;
            const int e0 = rw.t0 + rw.n0, e1 = e0 + rw.n1, e2 = e1 + rw.n2;
#pragma unroll 4
            for (int t = rw.t0 + p; t < e0; t += P) a0 += sw[t] * xl[soff[t]];
#pragma unroll 4
            for (int t = e0 + p; t < e1; t += P) a1 += sw[t] * xl[soff[t]];
#pragma unroll 4
            for (int t = e1 + p; t < e2; t += P) a2 += sw[t] * xl[soff[t]];
          }
          a0 = group_sum<P>(a0);
          a1 = group_sum<P>(a1);
          a2 = group_sum<P>(a2);
          if (ok && p == 0) {
            T v = a0;
            if (varnu) v += T(g.esc[k]) * a1 + T(g.eisc[k]) * a2;
            else v += a1 + a2;
            ts[rw.out * arr_t + il - sy] = bv - v;
          }
        }
      });
    }
    __syncthreads();
    // ---- xi Gauss-Seidel sweeps on A u = tmp_u (forward, and backward for A_s)
    int prev = -1;
    for (int sw_ = 0; sw_ < a.xi; ++sw_) {
      for (int pass = 0; pass < (a.ahat == HHG_AHAT_S ? 2 : 1); ++pass) {
        for (int pi = 0; pi < nph; ++pi) {
          const int ph = pass == 0 ? pi : nph - 1 - pi;
          if (ph == prev) continue;
          prev = ph;
          if (wbase < sd[ph].total) {
            const PhaseDesc d = sd[ph];
            const int grp = ph < 4 ? 0 : ph - 3, colour = ph < 4 ? ph : -1;
            const int t0 = srowA[grp].t0, t1 = t0 + srowA[grp].n1;
            const T inv_diag = sdiag[grp];
            with_lanes(d.lp, [&](auto lpc) {
              constexpr int LP = decltype(lpc)::value, P = 1 << LP;
              for (int q = tid; q < d.total; q += nthr) {
                const int inst = q >> LP, p = q & (P - 1);
                int i = 0, j = 0, k = d.kf;
                bool ok = false;
                if (inst < d.ninst) {
                  const int kk = qdiv(inst, d.m0), rem = inst - kk * d.d0, jj = qdiv(rem, d.m1);
                  const int ii = rem - jj * d.d1;
                  j = d.j0 + jj;
                  k += kk;
                  i = colour >= 0 ? 1 + ((colour - j - k - 1) & 3) + 4 * ii : d.i0 + ii;
                  ok = i <= g.nx - 1;
                }
                const int kl = k - kb;
                const int il = (i + 1) + (j + 1) * sx + (kl + 1) * sy;
                T a0 = T(0), a1 = T(0), a2 = T(0);
                if (ok) {
                  const T* us = xs + il;
#pragma unroll 4
                  for (int t = t0 + 1 + p; t < t1; t += P) {   // the diagonal is the first term
                    const T wt = sw[t];
                    const int o = soff[t];
                    a0 += wt * us[o];
                    a1 += wt * us[o + csl];
                    a2 += wt * us[o + 2 * csl];
                  }
                }
                a0 = group_sum<P>(a0);
                a1 = group_sum<P>(a1);
                a2 = group_sum<P>(a2);
                if (ok && p == 0) {
                  const T einv = varnu ? T(g.eisc[k]) : T(1);
                  const int ol = grp * arr_l + il, ot = grp * arr_t + il - sy;
                  store(ol, kl, (ts[ot] * einv - a0) * inv_diag);
                  store(ol + csl, kl, (ts[ot + cst] * einv - a1) * inv_diag);
                  store(ol + 2 * csl, kl, (ts[ot + 2 * cst] * einv - a2) * inv_diag);
                }
              }
            });
          }
          bar();
        }
      }
    }
    // ---- pressure step: tmp_p = g - (B u - C p) at every pressure site,
    // then p -= omega M_L^{-1} tmp_p
    if (wbase < sd[nph + 1].total) {
      const PhaseDesc d = sd[nph + 1];
      const ResRow& rw = tb.BC;
      with_lanes(d.lp, [&](auto lpc) {
        constexpr int LP = decltype(lpc)::value, P = 1 << LP;
        for (int q = tid; q < d.total; q += nthr) {
          const int inst = q >> LP, p = q & (P - 1);
          const bool valid = inst < d.ninst;
          int i = 0, j = 0, kl = 0;
          if (valid) {
            kl = qdiv(inst, d.m0);
            const int rem = inst - kl * d.d0;
            j = qdiv(rem, d.m1);
            i = rem - j * d.d1;
          }
          const int k = kb + kl;
          const bool bnd = i == 0 || j == 0 || k == 0 || i == g.nx || j == g.ny || k == g.nz;
          const bool comp = valid && (!bnd || rw.all);
          const int il = (i + 1) + (j + 1) * sx + (kl + 1) * sy;
          const int64_t ig = int64_t(i + 1) + int64_t(j + 1) * sx + int64_t(k + 1) * sy;
          const T bv = (comp && p == 0) ? __ldg(b + int64_t(rw.out) * g.arr + ig) : T(0);
          T a0 = T(0), a1 = T(0), a2 = T(0);
          if (comp) {
            const T* xl = xs + il;
            const int e0 = rw.t0 + rw.n0, e1 = e0 + rw.n1, e2 = e1 + rw.n2;
#pragma unroll 4
            for (int t = rw.t0 + p; t < e0; t += P) a0 += sw[t] * xl[soff[t]];
#pragma unroll 4
            for (int t = e0 + p; t < e1; t += P) a1 += sw[t] * xl[soff[t]];
            if (!bnd) {
#pragma unroll 4
              for (int t = e1 + p; t < e2; t += P) a2 += sw[t] * xl[soff[t]];
            } else {
              for (int t = rw.bs + p; t < rw.bs + rw.bn; t += P) {
                const DTermB tm = bc_op.bterms[t];
                const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
                if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
                a2 += bw<T>(bc_op, t) * xs[tm.arr * arr_l + il + tm.off];
              }
            }
          }
          a0 = group_sum<P>(a0);
          a1 = group_sum<P>(a1);
          a2 = group_sum<P>(a2);
          if (valid && p == 0) {
            T v = a0;
            if (varnu) v += T(g.esc[k]) * a1 + T(g.eisc[k]) * a2;
            else v += a1 + a2;
            ts[rw.out * arr_t + il - sy] = comp ? bv - v : T(0);
          }
        }
      });
    }
    bar();                                         // the neighbours have read the old halo pressures
    for (int r = tid; r < nk * sy; r += nthr) {    // owned planes, zero ring included (stays 0)
      const int kl = qdiv(r, msy);
      store(pol + sy + r, kl, xs[pol + sy + r] - mls[r] * ts[pot + r]);
    }
    bar();
  }
  // owned planes back to global memory
  {
    const int span = nk * sy;
    for (int q = tid; q < NA * span; q += nthr) {
      const int ar = q / span, r = q - ar * span;
      xg[int64_t(ar) * g.arr + int64_t(kb + 1) * sy + r] = xs[ar * arr_l + sy + r];
    }
  }
}

template <class T>
__global__ void __launch_bounds__(kResidentThreads)
    k_uzawa_resident(Geo g, int arr_l, int arr_t, T* xg, const T* __restrict__ b, const double* __restrict__ inv_ml,
                     const __grid_constant__ SmallArgs a, OpDev bc_op, const __grid_constant__ ResTabs<T> tb) {
  uzawa_resident_body<T>(g, arr_l, arr_t, xg, b, inv_ml, a, bc_op, tb);
}

template <class T>
struct ResA { Geo g; int arr_l, arr_t; T* xg; const T* b; const double* inv_ml; SmallArgs a; OpDev bc_op;
              const ResTabs<T>* tb; };
// every cluster of the merged grid belongs to one item (items start at
// multiples of the cluster size)
template <class T>
__global__ void __launch_bounds__(kResidentThreads) kb_uzawa_resident(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<ResA<T>>(items, n, bid, gd);
  const ResA<T>& r = it.a;
  uzawa_resident_body<T>(r.g, r.arr_l, r.arr_t, r.xg, r.b, r.inv_ml, r.a, r.bc_op, *r.tb);
}

template <class T> constexpr int prec_of() { return sizeof(T) == 8 ? HHG_FP64 : HHG_FP32; }

void fill_config(cudaLaunchConfig_t& cfg, cudaLaunchAttribute* attr, int C, int threads, size_t smem,
                 cudaStream_t s) {
  cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(threads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
}

template <class T>
bool feasible_impl(const Geo& g, int C) {
  if (C < 1 || C > kResidentMaxCtas || C > g.nz + 1) return false;
  // instance counts and divisors of a phase stay below 2^16 (qdiv)
  const int64_t planes = (g.nz + 1 + C - 1) / C;
  if (3 * int64_t(g.G) * (g.nx + 1) * (g.ny + 1) * planes >= 65536 || planes * g.sy >= 65536) return false;
  const size_t smem = resident_smem(g, C, prec_of<T>());
  if (smem > kResidentSmemMax) return false;
  auto fn = k_uzawa_resident<T>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kResidentSmemMax)) != cudaSuccess ||
      cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, C, kResidentThreads, smem, nullptr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return n > 0;
}

}  // namespace

int64_t resident_arr(const Geo& g, int ctas) {
  const int64_t nzp = g.nz + 1;
  const int64_t planes = (nzp + ctas - 1) / ctas + 2;
  return (planes * g.sy + 3) / 4 * 4;
}

int64_t resident_arr_t(const Geo& g, int ctas) {
  const int64_t nzp = g.nz + 1;
  return (((nzp + ctas - 1) / ctas) * g.sy + 3) / 4 * 4;
}

size_t resident_smem(const Geo& g, int ctas, int prec) {
  const size_t es = prec == HHG_FP64 ? 8 : 4;
  const size_t na = size_t(3 * g.G + 1);
  return (na * size_t(resident_arr(g, ctas)) + (na + 1) * size_t(resident_arr_t(g, ctas))) * es +
         size_t(kResMaxTerms) * (es + 4);
}

bool resident_feasible(int prec, const Geo& g, int ctas) {
  return prec == HHG_FP64 ? feasible_impl<double>(g, ctas) : feasible_impl<float>(g, ctas);
}

template <class T>
int uzawa_resident(const Geo& g, int ctas, int threads, T* x, const T* b, const double* inv_ml, const SmallArgs& a,
                   const OpDev& bc_op, const ResTabs<T>& tabs, cudaStream_t s) {
  if (threads < 128 || threads > kResidentThreads || threads % 32) return -1;
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  fill_config(cfg, attr, ctas, threads, resident_smem(g, ctas, prec_of<T>()), s);
  const int arr_l = int(resident_arr(g, ctas)), arr_t = int(resident_arr_t(g, ctas));
  if (g_rec) {
    const ResTabs<T>* dt = static_cast<const ResTabs<T>*>(g_rec->table(&tabs, sizeof(ResTabs<T>)));
    g_rec->add(reinterpret_cast<const void*>(kb_uzawa_resident<T>), dim3(ctas), dim3(threads), cfg.dynamicSmemBytes,
               ctas, ResA<T>{g, arr_l, arr_t, x, b, inv_ml, a, bc_op, dt});
    return dt ? 0 : -1;
  }
  ++g_launches;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_uzawa_resident<T>, g, arr_l, arr_t, x, b, inv_ml, a, bc_op, tabs);
  return e == cudaSuccess ? 0 : -1;
}

template int uzawa_resident<double>(const Geo&, int, int, double*, const double*, const double*, const SmallArgs&,
                                    const OpDev&, const ResTabs<double>&, cudaStream_t);
template int uzawa_resident<float>(const Geo&, int, int, float*, const float*, const double*, const SmallArgs&,
                                   const OpDev&, const ResTabs<float>&, cudaStream_t);

}  // namespace hhg
