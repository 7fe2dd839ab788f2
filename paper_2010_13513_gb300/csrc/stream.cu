// Streaming stencil rows: y = calA x and r = b - calA x over all rows of the
// operator (Eq. stokes-discrete), and the B^T and (B, -C) rows of the inexact
// Uzawa smoother (Sec. 3.2), on levels large enough to fill the GPU.
//
// Data reuse.  In the Kuhn-lattice layout an input value x(a, site) is read
// by the rows of every DoF group at about 27 neighbouring sites, so a kernel
// that loads every term on its own moves each input value from L2 into the SM
// many times.  Here a block owns M consecutive positions of the flattened
// (i, j) plane (M = V x threads; a thread owns V = 2 or 4 consecutive
// positions, one aligned vector, since the j pitch sx is a multiple of four)
// and a run of consecutive k planes, and marches through the run plane by
// plane:
//   * planes k-1, k, k+1 of the staged input arrays sit in a ring of four
//     shared-memory buffers (positions [m0 - sx - 4, m0 + M + sx + 4) of each
//     plane: the tile plus one lattice row and one quad of halo), and the
//     fourth buffer is filled with plane k+2 by cp.async while plane k is
//     evaluated, so every input value crosses from HBM/L2 once per pass;
//   * a thread loads each line (array, dj, dk) of its stencil footprint once
//     per plane -- one vector shared load of its V values and the i-1 / i+V
//     neighbours the line's terms need (V = 2: a scalar shared load each;
//     V = 4: from the neighbouring lanes by shuffles) -- and applies every
//     term of every row that reads that line to its V sites from registers.
// The plan (which arrays a pass stages, which rows it evaluates, the terms of
// each line with their row, segment and weight index) is emitted at build
// time by gen_structure.cpp from the stencil builder: every term is a
// compile-time register operation with a constant-bank weight.  Operators
// that read more than nine arrays (P2-P1: the full operator and B u - C p)
// take one launch per velocity component; the pressure row's first pass
// writes it and the later passes add their terms to it.
//
// Work split: the grid is one wave of blocks (the blocks that fit on the GPU
// at once); the (tile, plane) pairs of a pass, tile by tile, are cut into
// equal runs, one per block, so no block waits for a second wave.
//
// Rows on the domain boundary: velocity Dirichlet rows are 0; pressure rows
// keep the merged B terms (exact for inputs with zero Dirichlet velocity
// entries) and take their C terms from the clipped stencil of their boundary
// class (whether each of i, j, k lies on a low face, inside or on a high
// face: 27 classes), whose weights the library sums from the per-cube terms
// of the generic tables.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <utility>

#include "batch.h"
#include "fast.h"
#include "internal.h"
#include "kernels.h"
#include "stream.h"
#include "structure.inc"

namespace hhg {
namespace {

// ------------------------------------------------------------ cp.async
__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// V consecutive values of global memory (V x sizeof(T) bytes, aligned)
template <int V, class T>
__device__ __forceinline__ void gload(const T* p, T (&v)[V]) {
  if constexpr (sizeof(T) == 4 && V == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else if constexpr (sizeof(T) == 4) {
    const float2 q = *reinterpret_cast<const float2*>(p);
    v[0] = q.x; v[1] = q.y;
  } else {
#pragma unroll
    for (int h = 0; h < V / 2; ++h) {
      const double2 q = reinterpret_cast<const double2*>(p)[h];
      v[2 * h] = q.x; v[2 * h + 1] = q.y;
    }
  }
}
template <int V, class T>
__device__ __forceinline__ void gstore(T* p, const T (&v)[V]) {
  if constexpr (sizeof(T) == 4 && V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int h = 0; h < V / 2; ++h) reinterpret_cast<double2*>(p)[h] = make_double2(v[2 * h], v[2 * h + 1]);
  }
}

// ------------------------------------------------------ compile-time plan
template <class SPT, int Q>
constexpr int pass_e0() { return SPT::lines[SPT::passes[Q].l0].e0; }
template <class SPT, int Q>
constexpr int pass_e1() {
  return SPT::lines[SPT::passes[Q].l0 + SPT::passes[Q].nl - 1].e0 +
         SPT::lines[SPT::passes[Q].l0 + SPT::passes[Q].nl - 1].ne;
}
// whether part P of pass Q has C terms (segment 2)
template <class SPT, int Q, int P>
constexpr bool part_has_c() {
  for (int e = pass_e0<SPT, Q>(); e < pass_e1<SPT, Q>(); ++e)
    if (SPT::terms[e].part == P && SPT::terms[e].seg == 2) return true;
  return false;
}
// shared-memory slot of input array A in pass Q (-1 if not staged)
template <class SPT, int Q, int A>
constexpr int slot_of() {
  for (int a = 0; a < SPT::passes[Q].na; ++a)
    if (SPT::arrs[SPT::passes[Q].a0 + a] == A) return a;
  return -1;
}

template <int OG> struct Par {
  static constexpr int ox = OG == 1 || OG == 4 || OG == 5 || OG == 7;
  static constexpr int oy = OG == 2 || OG == 4 || OG == 6 || OG == 7;
  static constexpr int oz = OG == 3 || OG == 5 || OG == 6 || OG == 7;
};

// accumulators of a pass: row r = 3 * part + segment, V sites each
template <class T, int NA, int V> struct Acc {
  T a[NA][V];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int r = 0; r < NA; ++r)
#pragma unroll
      for (int s = 0; s < V; ++s) a[r][s] = T(0);
  }
  __device__ __forceinline__ void get(int r, T (&v)[V]) const {
#pragma unroll
    for (int s = 0; s < V; ++s) v[s] = a[r][s];
  }
};

// ----------------------------------------------------------- term evaluation
// with a constant viscosity the first two segments of a row (unscaled) share
// one accumulator; the C terms (segment 2) keep their own, which the clipped
// boundary stencil replaces on boundary pressure rows.  Every term is four
// FMAs with the weight from the constant bank.
// With a constant viscosity the weights are compile-time immediates: those of
// h = 1 (SPT::wref), the pressure values scaled by h as they are loaded and
// the rows scaled at the end (B, B^T scale as h^2, A as h, C as h^3).
template <class SPT, int E, int VARNU, class T, class Tab, int NA, int V>
__device__ __forceinline__ void term_fma(const T (&w)[V + 2], Acc<T, NA, V>& acc, const Tab& tab) {
  constexpr gen::TermE te = SPT::terms[E];
  constexpr int a = 3 * te.part + (VARNU || te.seg == 2 ? te.seg : 0);
  T wt;
  if constexpr (VARNU) {
    wt = tab.w[te.t];
  } else {
    constexpr double wd = SPT::wref[te.t];
    wt = T(wd);
  }
#pragma unroll
  for (int s = 0; s < V; ++s) acc.a[a][s] = fma(wt, w[te.di + 1 + s], acc.a[a][s]);
}

template <class SPT, int E0, int VARNU, class T, class Tab, int NA, int V, int... I>
__device__ __forceinline__ void line_terms(const T (&w)[V + 2], Acc<T, NA, V>& acc, const Tab& tab,
                                           std::integer_sequence<int, I...>) {
  (term_fma<SPT, E0 + I, VARNU>(w, acc, tab), ...);
}

// shared-memory buffer of plane kp (ring of four)
__device__ __forceinline__ int64_t buf_of(int kp, int64_t bufsz) { return ((kp + 1) & 3) * bufsz; }

// shared-memory loads with 32-bit shared addresses: the thread's V values
// (into w[1 .. V]), and one value
template <int V>
__device__ __forceinline__ void lds_vec(uint32_t a, float (&w)[V + 2]) {
  if constexpr (V == 4)
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(w[1]), "=f"(w[2]), "=f"(w[3]), "=f"(w[4]) : "r"(a));
  else
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(w[1]), "=f"(w[2]) : "r"(a));
}
template <int V>
__device__ __forceinline__ void lds_vec(uint32_t a, double (&w)[V + 2]) {
#pragma unroll
  for (int h = 0; h < V / 2; ++h)
    asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(w[2 * h + 1]), "=d"(w[2 * h + 2]) : "r"(a + 16 * h));
}
__device__ __forceinline__ void lds1(uint32_t a, float& v) { asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a)); }
// one value loaded by one lane only (predicated, no branch)
__device__ __forceinline__ void lds_if(bool on, uint32_t a, float& v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n @q ld.shared.f32 %0, [%2];\n}"
               : "+f"(v) : "r"(unsigned(on)), "r"(a));
}
__device__ __forceinline__ void lds_if(bool on, uint32_t a, double& v) {
  asm volatile("{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n @q ld.shared.f64 %0, [%2];\n}"
               : "+d"(v) : "r"(unsigned(on)), "r"(a));
}
__device__ __forceinline__ void lds1(uint32_t a, double& v) { asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a)); }

// one line (slot, dj, dk): the thread's V values and the neighbours i - 1
// and i + V that the line's terms need (the staged line holds them for every
// lane), then every term of the line.  pb[dk + 1] is
// the shared address of the thread's values in slot 0 of plane k + dk; lwb,
// sxb: the slot and row strides in bytes.
template <class SPT, int L, int VARNU, int PSLOT, class T, class Tab, int NA, int V>
__device__ __forceinline__ void eval_line(const uint32_t (&pb)[3], int lwb, int sxb, int lane, T hs,
                                          Acc<T, NA, V>& acc, const Tab& tab) {
  constexpr gen::LineT ln = SPT::lines[L];
  constexpr int es = int(sizeof(T));
  const uint32_t a = pb[ln.dk + 1] + uint32_t(ln.slot * lwb + ln.dj * sxb);
  T w[V + 2];
  lds_vec<V>(a, w);
  if constexpr (V == 2) {
    // lanes two values apart: a scalar load per neighbour (two-way bank
    // conflict) issues fewer instructions than a shuffle
    if constexpr (ln.lmin < 0) lds1(a - es, w[0]);
    if constexpr (ln.lmax > 0) lds1(a + V * es, w[V + 1]);
  } else {
    // lanes four values apart: the neighbours from the neighbouring lanes by
    // shuffles, and the block's end values by one lane's load (a scalar load
    // per lane would be a four-way bank conflict)
    if constexpr (ln.lmin < 0) {
      T v = __shfl_up_sync(0xffffffffu, w[V], 1);
      lds_if(lane == 0, a - es, v);
      w[0] = v;
    }
    if constexpr (ln.lmax > 0) {
      T v = __shfl_down_sync(0xffffffffu, w[1], 1);
      lds_if(lane == 31, a + V * es, v);
      w[V + 1] = v;
    }
  }
  if constexpr (!VARNU && ln.slot == PSLOT) {
#pragma unroll
    for (int s = 0; s < V + 2; ++s) w[s] *= hs;
  }
  line_terms<SPT, ln.e0, VARNU>(w, acc, tab, std::make_integer_sequence<int, ln.ne>{});
}

template <class SPT, int L0, int VARNU, int PSLOT, class T, class Tab, int NA, int V, int... I>
__device__ __forceinline__ void eval_lines(const uint32_t (&pb)[3], int lwb, int sxb, int lane, T hs,
                                           Acc<T, NA, V>& acc, const Tab& tab, std::integer_sequence<int, I...>) {
  (eval_line<SPT, L0 + I, VARNU, PSLOT>(pb, lwb, sxb, lane, hs, acc, tab), ...);
}

// C terms of a boundary pressure row at site (i, j, k), staged position lf:
// the clipped stencil of the site's boundary class applied to the pressure
// values in shared memory (slot SLOTP)
template <class SPT, int SLOTP, class T, class Tab, int... O>
__device__ __forceinline__ T boundary_c(const Geo& g, const T* sm, int64_t bufsz, int lw, int lf, int i, int j, int k,
                                        const Tab& tab, std::integer_sequence<int, O...>) {
  const int cls = (i == 0 ? 0 : i == g.nx ? 2 : 1) + 3 * (j == 0 ? 0 : j == g.ny ? 2 : 1) +
                  9 * (k == 0 ? 0 : k == g.nz ? 2 : 1);
  const T* wc = tab.wc + cls * SPT::NCB;
  T a = T(0);
  ((a += wc[O] * sm[buf_of(k + SPT::cbo[O].dk, bufsz) + SLOTP * lw + lf + SPT::cbo[O].dj * g.sx + SPT::cbo[O].di]),
   ...);
  return a;
}

// --------------------------------------------------------------- outputs
// where the thread's sites lie, for the output groups of both parities of
// each index (group offset o = 0: lattice sites 0 .. n; o = 1: 0 .. n - 1,
// never on a face): the i flags once per tile, the k flags once per plane
template <int V>
struct SiteFlags {
  bool in0[V], in1[V];   // 0 <= i <= nx, 0 <= i <= nx - 1
  bool ib[V];            // i == 0 or i == nx
  bool jin0, jin1, jb;   // the same for j
  bool kin1, kb;         // k <= nz - 1; k == 0 or k == nz (k <= nz always)
};
// the rows of part P at the thread's V sites (positions fk .. fk + V - 1 of
// the k plane: coarse indices (i0 .. i0 + V - 1, j, k)), written to y as one
// vector.  Positions outside the group's sites (the halo column, the row
// padding) and Dirichlet velocity rows are written as 0: halo, padding and
// Dirichlet entries of every vector are 0, so the vector store never changes
// them.
template <class SPT, int Q, int P, int VARNU, int PSLOT, class T, int MODE, class Tab, int NA, int V>
__device__ __forceinline__ void store_part(const Geo& g, const T* __restrict__ b, T* __restrict__ y, const T* sm,
                                           int64_t bufsz, int lw, int lf, int k, int i0, int j, int64_t fk, T es, T eis,
                                           const Acc<T, NA, V>& acc, const Tab& tab, const SiteFlags<V>& sf) {
  constexpr gen::PartT pt = SPT::parts[SPT::passes[Q].p0 + P];
  constexpr bool HAS_C = part_has_c<SPT, Q, P>();
  using PP = Par<pt.og>;
  // the row's DoF at doubled position 2 (i, j, k) + (ox, oy, oz): an odd
  // component never lies on a face
  if (!(PP::oy ? sf.jin1 : sf.jin0) || (PP::oz && !sf.kin1)) return;
  const bool bjk = (PP::oy ? false : sf.jb) || (PP::oz ? false : sf.kb);
  T a0[V], a1[V], a2[V], v[V];
  acc.get(3 * P, a0);
  if (VARNU) acc.get(3 * P + 1, a1);
  if (HAS_C) acc.get(3 * P + 2, a2);
  // constant viscosity: the scale of the row (h for velocity rows, h^2 for
  // pressure rows; the pressure values entered scaled by h)
  const T hs = pt.all ? T(g.h) * T(g.h) : T(g.h);
  bool keep[V];
#pragma unroll
  for (int s = 0; s < V; ++s) {
    v[s] = a0[s];
    if (VARNU) v[s] += es * a1[s];
    if (HAS_C) v[s] += VARNU ? eis * a2[s] : a2[s];
    if (!VARNU) v[s] *= hs;
    const int i = i0 + s;
    const bool bnd = bjk || (PP::ox ? false : sf.ib[s]);
    keep[s] = (PP::ox ? sf.in1[s] : sf.in0[s]) && (pt.all || !bnd);
    if constexpr (HAS_C) {
      if (keep[s] && bnd) {                            // boundary pressure row: clipped C stencil
        static_assert(PSLOT >= 0, "the pressure array is staged with the C terms");
        const T c = boundary_c<SPT, PSLOT, T>(g, sm, bufsz, lw, lf + s, i, j, k, tab,
                                              std::make_integer_sequence<int, SPT::NCB>{});
        v[s] = VARNU ? a0[s] + es * a1[s] + eis * c : hs * a0[s] + c;
      }
    }
  }
  const int64_t iy = int64_t(pt.out) * g.arr + fk;
  T o[V];
  if (pt.first) {
    if (MODE == MODE_RES) {
      T bb[V];
      gload<V>(b + iy, bb);
#pragma unroll
      for (int s = 0; s < V; ++s) o[s] = keep[s] ? bb[s] - v[s] : T(0);
    } else {
#pragma unroll
      for (int s = 0; s < V; ++s) o[s] = keep[s] ? v[s] : T(0);
    }
  } else {
    T c[V];
    gload<V>(y + iy, c);
#pragma unroll
    for (int s = 0; s < V; ++s) o[s] = keep[s] ? (MODE == MODE_RES ? c[s] - v[s] : c[s] + v[s]) : c[s];
  }
  gstore<V>(y + iy, o);
}

template <class SPT, int Q, int VARNU, int PSLOT, class T, int MODE, class Tab, int NA, int V, int... I>
__device__ __forceinline__ void store_parts(const Geo& g, const T* __restrict__ b, T* __restrict__ y, const T* sm,
                                            int64_t bufsz, int lw, int lf, int k, int i0, int j, int64_t fk, T es,
                                            T eis, const Acc<T, NA, V>& acc, const Tab& tab, const SiteFlags<V>& sf,
                                            std::integer_sequence<int, I...>) {
  (store_part<SPT, Q, I, VARNU, PSLOT, T, MODE>(g, b, y, sm, bufsz, lw, lf, k, i0, j, fk, es, eis, acc, tab, sf), ...);
}

// cp.async of plane kp of the pass's arrays (array slot A at buf + A lw);
// chunks outside the vector are skipped (they feed only positions whose rows
// are not stored)
template <class SPT, int Q, class T, int... A>
__device__ __forceinline__ void stage_plane(const T* __restrict__ x, T* buf, int64_t pbase, int64_t arr, int64_t vlen,
                                            int lw, int nch, int tid, int nt, std::integer_sequence<int, A...>) {
  constexpr int VE = 16 / int(sizeof(T));
  auto one = [&](int slot, int64_t base) {
    T* dst = buf + slot * lw;
    if (base >= 0 && base + lw <= vlen) {            // the whole line lies in the vector (all but the ends)
      const T* src = x + base;
      for (int c = tid; c < nch; c += nt) cp16(dst + c * VE, src + c * VE);
    } else {
      for (int c = tid; c < nch; c += nt) {
        const int64_t e = base + int64_t(c) * VE;
        if (e >= 0 && e + VE <= vlen) cp16(dst + c * VE, x + e);
      }
    }
  };
  (one(A, int64_t(std::integral_constant<int, SPT::arrs[SPT::passes[Q].a0 + A]>::value) * arr + pbase), ...);
}

// ------------------------------------------------------------------ a pass
// grid: one wave of blocks.  kc > 0 (lockstep): block b takes tile b % tiles
// and planes [c kc, (c + 1) kc) with c = b / tiles, so that blocks on
// neighbouring tiles march through the same planes at the same time and the
// halo rows they share come from L2.  kc = 0 (balanced): block b takes the
// (tile, plane) pairs [b U / grid, (b + 1) U / grid) of the U = tiles x
// (nz + 1) pairs, tile by tile.  On each tile a block marches through its
// planes.
// (bx, gx: the block's index and the grid size; the plain kernel passes
// blockIdx.x and gridDim.x, the batched one the values of its work item)
template <int DISC, int VARNU, int OP, int Q, class T, int MODE, int V, class Tab>
__device__ __forceinline__ void stream_body(const unsigned bx, const unsigned gx, const Geo& g,
                                            const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y,
                                            int lw, int64_t units, int64_t tiles, int kc, const Tab& tab) {
  using SPT = gen::SP<DISC, VARNU, OP>;
  constexpr gen::PassT ps = SPT::passes[Q];
  constexpr int PSLOT = slot_of<SPT, Q, (DISC == 2 ? 24 : 3)>();
  constexpr int VE = 16 / int(sizeof(T));
  extern __shared__ __align__(16) unsigned char stream_smem[];
  T* sm = reinterpret_cast<T*>(stream_smem);
  const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(stream_smem));
  const int tid = threadIdx.x, lane = tid & 31, nt = blockDim.x;
  const int M = V * nt, sx = g.sx;
  const int nk = g.nz + 1;
  const int nch = lw / VE;
  const int64_t vlen = int64_t(3 * g.G + 1) * g.arr;
  const int64_t bufsz = int64_t(SPT::NAMAX) * lw;
  const int lf = V * tid + sx + 4;                   // the thread's sites in a staged line
  int64_t u, uend;
  if (kc > 0) {
    const int64_t t = bx % tiles, c = bx / tiles;
    u = t * nk + min(int64_t(nk), c * kc);
    uend = t * nk + min(int64_t(nk), (c + 1) * kc);
  } else {
    u = int64_t(bx) * units / gx;
    uend = int64_t(bx + 1) * units / gx;
  }
#pragma unroll 1
  while (u < uend) {
    const int64_t tile = u / nk;
    const int k0 = int(u - tile * nk);
    const int k1 = int(k0 + min(int64_t(nk - k0), uend - u));
    u += k1 - k0;
    const int64_t m0 = int64_t(sx) + tile * M;
    const int64_t gbase = m0 - sx - 4;
    const int64_t f = m0 + V * tid;                    // the thread's first site
    const int j = int(f / sx) - 1;
    const int i0 = int(f - int64_t(j + 1) * sx) - 1;
    SiteFlags<V> sf;
#pragma unroll
    for (int s = 0; s < V; ++s) {
      const int i = i0 + s;
      sf.in0[s] = i >= 0 && i <= g.nx;
      sf.in1[s] = i >= 0 && i <= g.nx - 1;
      sf.ib[s] = i == 0 || i == g.nx;
    }
    sf.jin0 = j >= 0 && j <= g.ny;
    sf.jin1 = j >= 0 && j <= g.ny - 1;
    sf.jb = j == 0 || j == g.ny;
    auto load = [&](int kp) {
      stage_plane<SPT, Q>(x, sm + buf_of(kp, bufsz), int64_t(kp + 1) * g.sy + gbase, g.arr, vlen, lw, nch, tid, nt,
                          std::make_integer_sequence<int, ps.na>{});
    };
    __syncthreads();                                   // the previous run no longer reads the ring
    load(k0 - 1);
    cp_commit();
    load(k0);
    cp_commit();
    load(k0 + 1);
    cp_commit();
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
      if (k + 1 < k1) load(k + 2);
      cp_commit();
      cp_wait1();                                      // planes k-1, k, k+1 are in place (this thread's copies)
      __syncthreads();                                 // ... and every thread's
      Acc<T, 3 * ps.np, V> acc;
      acc.zero();
      const uint32_t pb[3] = {sbase + uint32_t(buf_of(k - 1, bufsz) + lf) * uint32_t(sizeof(T)),
                              sbase + uint32_t(buf_of(k, bufsz) + lf) * uint32_t(sizeof(T)),
                              sbase + uint32_t(buf_of(k + 1, bufsz) + lf) * uint32_t(sizeof(T))};
      eval_lines<SPT, ps.l0, VARNU, PSLOT>(pb, lw * int(sizeof(T)), sx * int(sizeof(T)), lane, T(g.h), acc, tab,
                                           std::make_integer_sequence<int, ps.nl>{});
      T es = T(1), eis = T(1);
      if (VARNU) {
        es = T(g.esc[k]);
        eis = T(g.eisc[k]);
      }
      sf.kin1 = k <= g.nz - 1;
      sf.kb = k == 0 || k == g.nz;
      store_parts<SPT, Q, VARNU, PSLOT, T, MODE>(g, b, y, sm, bufsz, lw, lf, k, i0, j, int64_t(k + 1) * g.sy + f, es,
                                                 eis, acc, tab, sf, std::make_integer_sequence<int, ps.np>{});
      __syncthreads();                                 // plane k-1's buffer is refilled next
    }
    cp_wait0();
  }
}

template <int DISC, int VARNU, int OP, int Q, class T, int MODE, int V, class Tab>
__global__ void __launch_bounds__(256, 2)
    k_stream(Geo g, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ y, int lw, int64_t units,
             int64_t tiles, int kc, const __grid_constant__ Tab tab) {
  stream_body<DISC, VARNU, OP, Q, T, MODE, V>(blockIdx.x, gridDim.x, g, x, b, y, lw, units, tiles, kc, tab);
}

// one pass as a work item of a merged batch launch (the table as a device copy)
template <class T, class Tab>
struct StreamA { Geo g; const T* x; const T* b; T* y; int lw; int64_t units, tiles; int kc; const Tab* tab; };
template <int DISC, int VARNU, int OP, int Q, class T, int MODE, int V, class Tab>
__global__ void __launch_bounds__(256, 2) kb_stream(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<StreamA<T, Tab>>(items, n, bid, gd);
  const StreamA<T, Tab>& a = it.a;
  stream_body<DISC, VARNU, OP, Q, T, MODE, V>(bid.x, gd.x, a.g, a.x, a.b, a.y, a.lw, a.units, a.tiles, a.kc, *a.tab);
}

// --------------------------------------------------------- launch support
// parameter block of the streaming kernels of one operator
template <class T, int N, int NCB> struct STab {
  T w[N];                             // weights, in the order of the FastTab images
  T wc[NCB > 0 ? 27 * NCB : 1];       // clipped boundary C stencils per class
};

template <int DISC, int VARNU, int OP, class T>
using STabOf = STab<T, gen::S<DISC, VARNU, OP>::N, gen::SP<DISC, VARNU, OP>::NCB>;

size_t smem_bytes(int namax, const Geo& g, int threads, int v, size_t es) {
  return size_t(4) * namax * size_t(v * threads + 2 * g.sx + 8) * es;
}

// blocks of a kernel that fit on one SM, and the SM count (cached)
int blocks_per_sm(const void* fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t>, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto key = std::make_tuple(fn, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem) != cudaSuccess) {
    cudaGetLastError();
    n = 1;
  }
  cache[key] = n;
  return n;
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      n = 132;
    }
  }
  return n;
}

// grid of a pass: one wave of blocks (per_sm resident blocks per SM)
struct PassGrid {
  int64_t grid, units, tiles;
  int kc;
};
inline PassGrid pass_grid(const Geo& g, int per_sm, int M) {
  PassGrid p;
  p.tiles = (int64_t(g.ny + 1) * g.sx + M - 1) / M;
  const int nk = g.nz + 1;
  p.units = p.tiles * nk;
  const int64_t resident = int64_t(per_sm) * sm_count();
  p.grid = std::min<int64_t>(p.units, resident);
  p.kc = 0;
  // lockstep chunks if they fill at least 85 % of the resident blocks
  const int64_t chunks = resident / p.tiles;
  if (chunks >= 1 && p.tiles * chunks * 100 >= 85 * resident) {
    p.kc = int((nk + chunks - 1) / chunks);
    p.grid = p.tiles * ((nk + p.kc - 1) / p.kc);
  }
  return p;
}

#if !defined(HHG_STREAM_BATCHED)
template <int DISC, int VARNU, int OP, int Q, class T, int MODE, int V>
bool launch_pass(const Geo& g, const void* tab, const T* x, const T* b, T* y, int threads, cudaStream_t s) {
  using SPT = gen::SP<DISC, VARNU, OP>;
  using Tab = STabOf<DISC, VARNU, OP, T>;
  const Tab& tb = *static_cast<const Tab*>(tab);
  const size_t smem = smem_bytes(SPT::NAMAX, g, threads, V, sizeof(T));
  auto fn = k_stream<DISC, VARNU, OP, Q, T, MODE, V, Tab>;
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(fn), threads, smem);
  if (per_sm < 1) return false;
  const int M = V * threads;
  const PassGrid pg = pass_grid(g, per_sm, M);
  ++g_launches;
  fn<<<unsigned(pg.grid), threads, smem, s>>>(g, x, b, y, int(M + 2 * g.sx + 8), pg.units, pg.tiles, pg.kc, tb);
  return true;
}
#else
// the same pass as a work item of the batch being recorded (batch.h); the
// stream argument is unused
template <int DISC, int VARNU, int OP, int Q, class T, int MODE, int V>
bool launch_pass(const Geo& g, const void* tab, const T* x, const T* b, T* y, int threads, cudaStream_t) {
  using SPT = gen::SP<DISC, VARNU, OP>;
  using Tab = STabOf<DISC, VARNU, OP, T>;
  const size_t smem = smem_bytes(SPT::NAMAX, g, threads, V, sizeof(T));
  auto fn = kb_stream<DISC, VARNU, OP, Q, T, MODE, V, Tab>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStreamMaxSmem)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int per_sm = blocks_per_sm(reinterpret_cast<const void*>(fn), threads, smem);
  if (per_sm < 1) return false;
  const int M = V * threads;
  const PassGrid pg = pass_grid(g, per_sm, M);
  const Tab* dt = static_cast<const Tab*>(g_rec->table(tab, sizeof(Tab)));
  g_rec->add(reinterpret_cast<const void*>(fn), dim3(unsigned(pg.grid)), dim3(threads), smem, 1,
             StreamA<T, Tab>{g, x, b, y, int(M + 2 * g.sx + 8), pg.units, pg.tiles, pg.kc, dt});
  return true;
}
#endif

template <int DISC, int VARNU, int OP, class T, int MODE, int V, int... Q>
void launch_passes(const Geo& g, const void* tab, const T* x, const T* b, T* y, int threads, cudaStream_t s,
                   std::integer_sequence<int, Q...>) {
  (launch_pass<DISC, VARNU, OP, Q, T, MODE, V>(g, tab, x, b, y, threads, s), ...);
}

// sites per thread compiled in this translation unit (FP64: 4; FP32: 4, or
// 2 in the unit built with HHG_STREAM_V = 2)
#if defined(HHG_STREAM_V) && HHG_STREAM_V == 2
constexpr int kV = 2;
#else
constexpr int kV = 4;
#endif

template <int DISC, int VARNU, int OP, class T>
bool launch_stream(const Geo& g, const void* tab, int mode, const T* x, const T* b, T* y, int threads,
                   cudaStream_t s) {
  using SPT = gen::SP<DISC, VARNU, OP>;
  if ((threads != 64 && threads != 128 && threads != 256) || (g.sx & 3) || (g.arr & 3)) return false;
  // the thread's sites are read and written as vectors
  if ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(b)) & 15)
    return false;
  if (smem_bytes(SPT::NAMAX, g, threads, kV, sizeof(T)) > kStreamMaxSmem) return false;
  if (mode == MODE_SET)
    launch_passes<DISC, VARNU, OP, T, MODE_SET, kV>(g, tab, x, b, y, threads, s,
                                                    std::make_integer_sequence<int, SPT::NP>{});
  else
    launch_passes<DISC, VARNU, OP, T, MODE_RES, kV>(g, tab, x, b, y, threads, s,
                                                    std::make_integer_sequence<int, SPT::NP>{});
  return true;
}

#if !defined(HHG_STREAM_BATCHED)
template <int DISC, int VARNU, int OP, class T, int... Q>
void init_passes(std::integer_sequence<int, Q...>) {
  using Tab = STabOf<DISC, VARNU, OP, T>;
  ((cudaFuncSetAttribute(k_stream<DISC, VARNU, OP, Q, T, MODE_SET, kV, Tab>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStreamMaxSmem)),
    cudaFuncSetAttribute(k_stream<DISC, VARNU, OP, Q, T, MODE_RES, kV, Tab>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(kStreamMaxSmem))),
   ...);
}

template <int DISC, int VARNU, int OP, class T>
void init_stream() {
  init_passes<DISC, VARNU, OP, T>(std::make_integer_sequence<int, gen::SP<DISC, VARNU, OP>::NP>{});
}
#endif

// the parameter block from the weights (FastTab order) and the class sums of
// the boundary C stencils (27 x NCB, offsets in the order of cbo)
template <int DISC, int VARNU, int OP, class T>
void make_image(const std::vector<double>& w, const std::vector<double>& wc, std::vector<char>& out) {
  using SPT = gen::SP<DISC, VARNU, OP>;
  using Tab = STabOf<DISC, VARNU, OP, T>;
  out.assign(sizeof(Tab), 0);
  Tab* t = reinterpret_cast<Tab*>(out.data());
  const int N = gen::S<DISC, VARNU, OP>::N;
  for (int i = 0; i < N && i < int(w.size()); ++i) t->w[i] = T(w[i]);
  for (int i = 0; i < 27 * SPT::NCB && i < int(wc.size()); ++i) t->wc[i] = T(wc[i]);
}

template <int DISC, int VARNU, int OP>
void offsets_of(std::vector<int>& o) {
  using SPT = gen::SP<DISC, VARNU, OP>;
  o.clear();
  if constexpr (SPT::NCB > 0)
    for (int i = 0; i < SPT::NCB; ++i) {
      o.push_back(SPT::cbo[i].di);
      o.push_back(SPT::cbo[i].dj);
      o.push_back(SPT::cbo[i].dk);
    }
}

}  // namespace

#define HHG_STREAM_CASES(X) \
  X(1, 0, OP_FULL) X(1, 0, OP_BT) X(1, 0, OP_BC) X(1, 1, OP_FULL) X(1, 1, OP_BT) X(1, 1, OP_BC) \
  X(2, 0, OP_FULL) X(2, 0, OP_BT) X(2, 0, OP_BC) X(2, 1, OP_FULL) X(2, 1, OP_BT) X(2, 1, OP_BC)

#if defined(HHG_STREAM_BATCHED)
// the recorder of this translation unit's kernels (precision HHG_STREAM_ONLY,
// kV sites per thread): the passes become work items of the batch being
// recorded
template <class T, int V>
bool stream_rows_record_v(int disc, int varnu, int op, int mode, const Geo& g, const void* tab, const T* x,
                          const T* b, T* y, int threads) {
  static_assert(V == kV, "one site count per translation unit");
  if (mode != MODE_SET && mode != MODE_RES) return false;
#define HHG_S(D, V_, O) \
  if (disc == D && varnu == V_ && op == O) return launch_stream<D, V_, O, T>(g, tab, mode, x, b, y, threads, nullptr);
  HHG_STREAM_CASES(HHG_S)
#undef HHG_S
  return false;
}
#if defined(HHG_STREAM_ONLY) && HHG_STREAM_ONLY == 32
template bool stream_rows_record_v<float, kV>(int, int, int, int, const Geo&, const void*, const float*, const float*,
                                              float*, int);
#else
template bool stream_rows_record_v<double, kV>(int, int, int, int, const Geo&, const void*, const double*,
                                               const double*, double*, int);
#endif
#else
// the kernels of this translation unit (precision HHG_STREAM_ONLY, kV sites
// per thread); while a batch records, the batched units take the call
template <class T, int V>
bool stream_rows_v(int disc, int varnu, int op, int mode, const Geo& g, const void* tab, const T* x, const T* b, T* y,
                   int threads, cudaStream_t s) {
  static_assert(V == kV, "one site count per translation unit");
  if (g_rec) return stream_rows_record_v<T, V>(disc, varnu, op, mode, g, tab, x, b, y, threads);
  if (mode != MODE_SET && mode != MODE_RES) return false;
#define HHG_S(D, V_, O) \
  if (disc == D && varnu == V_ && op == O) return launch_stream<D, V_, O, T>(g, tab, mode, x, b, y, threads, s);
  HHG_STREAM_CASES(HHG_S)
#undef HHG_S
  return false;
}

template <class T, int V>
void stream_init_v() {
#define HHG_I(D, V_, O) init_stream<D, V_, O, T>();
  HHG_STREAM_CASES(HHG_I)
#undef HHG_I
}

#if defined(HHG_STREAM_ONLY) && HHG_STREAM_ONLY == 32
template bool stream_rows_v<float, kV>(int, int, int, int, const Geo&, const void*, const float*, const float*, float*,
                                       int, cudaStream_t);
template void stream_init_v<float, kV>();
#else
template bool stream_rows_v<double, kV>(int, int, int, int, const Geo&, const void*, const double*, const double*,
                                        double*, int, cudaStream_t);
template void stream_init_v<double, kV>();
#endif

#if !defined(HHG_STREAM_V) || HHG_STREAM_V != 2
template <class T>
bool stream_image(int disc, int varnu, int op, const std::vector<double>& w, const std::vector<double>& wc,
                  std::vector<char>& out) {
#define HHG_M(D, V, O) \
  if (disc == D && varnu == V && op == O) { make_image<D, V, O, T>(w, wc, out); return true; }
  HHG_STREAM_CASES(HHG_M)
#undef HHG_M
  return false;
}
#if defined(HHG_STREAM_ONLY) && HHG_STREAM_ONLY == 32
template bool stream_image<float>(int, int, int, const std::vector<double>&, const std::vector<double>&,
                                  std::vector<char>&);
#else
template bool stream_image<double>(int, int, int, const std::vector<double>&, const std::vector<double>&,
                                   std::vector<char>&);

bool stream_c_offsets(int disc, int varnu, int op, std::vector<int>& offsets) {
#define HHG_O(D, V, O) \
  if (disc == D && varnu == V && op == O) { offsets_of<D, V, O>(offsets); return true; }
  HHG_STREAM_CASES(HHG_O)
#undef HHG_O
  return false;
}

// FP32 rows take 2 or 4 sites per thread (two other translation units), FP64
// four
extern template bool stream_rows_v<float, 4>(int, int, int, int, const Geo&, const void*, const float*, const float*,
                                             float*, int, cudaStream_t);
extern template bool stream_rows_v<float, 2>(int, int, int, int, const Geo&, const void*, const float*, const float*,
                                             float*, int, cudaStream_t);
extern template void stream_init_v<float, 4>();
extern template void stream_init_v<float, 2>();

template <class T>
bool stream_rows(int disc, int varnu, int op, int mode, const Geo& g, const void* tab, const T* x, const T* b, T* y,
                 int threads, int sites, cudaStream_t s) {
  if constexpr (sizeof(T) == 4) {
    if (sites == 2) return stream_rows_v<T, 2>(disc, varnu, op, mode, g, tab, x, b, y, threads, s);
  }
  return stream_rows_v<T, 4>(disc, varnu, op, mode, g, tab, x, b, y, threads, s);
}
template <class T>
void stream_init() {
  stream_init_v<T, 4>();
  if constexpr (sizeof(T) == 4) stream_init_v<T, 2>();
}
template bool stream_rows<double>(int, int, int, int, const Geo&, const void*, const double*, const double*, double*,
                                  int, int, cudaStream_t);
template bool stream_rows<float>(int, int, int, int, const Geo&, const void*, const float*, const float*, float*, int,
                                 int, cudaStream_t);
template void stream_init<double>();
template void stream_init<float>();
#endif
#endif

#endif  // HHG_STREAM_BATCHED

}  // namespace hhg
