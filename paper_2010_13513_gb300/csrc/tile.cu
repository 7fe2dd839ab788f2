// Shared-memory-tiled stencil rows (FP32): y = calA x, r = b - calA x, and
// the B^T / (B, -C) residual rows of the smoother, on levels large enough to
// fill the GPU.
//
// In the Kuhn-lattice layout every input value x(a, site) is read by about 35
// row evaluations (the rows of all groups at the ~27 neighbouring sites), so
// reading each term from L1/L2 costs one load instruction with its address
// arithmetic and thrashes L1 with the neighbourhoods of up to 25 arrays.  Here
// a block owns a TI x TJ x TK tile of lattice sites and one block type of the
// operator: the rows that read the same input arrays (P2-P1 full operator: the
// 8 velocity rows of one component, reading that component's 8 group arrays
// and the pressure; the pressure row, reading the 24 velocity arrays).  The
// block copies the tile plus a one-site halo of exactly those arrays into
// shared memory with coalesced loads, then each thread evaluates its rows
// there: every term is one shared-memory load with a compile-time offset and
// one FMA with a constant-bank weight.  The row structure, the block types,
// the tile slot of every input array and the lattice offset of every term are
// emitted at build time by gen_structure.cpp from the stencil builder.  The
// tile is copied with cp.async (all copies of a block in flight at once).
// Measured on GB300 (event timing, L2 flushed): 197 us for the P2-P1 level-6
// apply against 89 us for the plain kernels, 1.27 ms against 0.70 ms for P1-P1
// level 7 -- the copy phase and the per-row bookkeeping cost more issue slots
// than the L1 re-reads they save -- so the plain kernels stay the default and
// the autotuner keeps these as a candidate.
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include "fast.h"
#include "internal.h"
#include "kernels.h"
#include "structure.inc"
#include "tile.h"

namespace hhg {
namespace {

constexpr int TI = 32, TJ = 4, TK = 4;           // owned sites per tile
constexpr int TX = TI + 2, TY = TJ + 2, TZ = TK + 2;
constexpr int VOL = TX * TY * TZ;                 // tile + halo, per input array
constexpr int kTileThreads = 256;

template <class PL, int t>
struct TermOff {                                  // tile offset of term t relative to its site
  static constexpr int v = PL::terms[t].slot * VOL + PL::terms[t].di + PL::terms[t].dj * TX + PL::terms[t].dk * TX * TY;
};

template <class PL, int T0, class T, class Tab, int... I>
__device__ __forceinline__ T tseg(const Tab& tab, const T* s, std::integer_sequence<int, I...>) {
  T a = T(0);
  ((a += tab.w[T0 + I] * s[TermOff<PL, T0 + I>::v]), ...);
  return a;
}

// per-cube evaluation of the third segment (C terms) of a boundary row, from
// global memory (boundary pressure rows under variable viscosity only)
__device__ __forceinline__ float tboundary_seg2(const Geo& g, const OpDev& op, int r, int i, int j, int k,
                                                const float* x, int64_t idx) {
  const DRow row = op.rows[r];
  float a = 0.f;
  for (int t = row.b0 + row.m0 + row.m1; t < row.b0 + row.m0 + row.m1 + row.m2; ++t) {
    const DTermB tm = op.bterms[t];
    const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
    if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
    a += __ldg(op.bw32 + t) * x[int64_t(tm.arr) * g.arr + idx + tm.off];
  }
  return a;
}

template <int DISC, int VARNU, int OP, int MODE, int R, class Tab>
__device__ __forceinline__ void tile_row(const Geo& g, int i, int j, int k, const float* s, const float* __restrict__ x,
                                         const float* __restrict__ b, float* __restrict__ y, float alpha,
                                         const OpDev& op, const Tab& tab) {
  using S = gen::S<DISC, VARNU, OP>;
  using PL = gen::P<DISC, VARNU, OP>;
  constexpr gen::RowS rw = S::rows[R];
  constexpr int ox = rw.og == 1 || rw.og == 4 || rw.og == 5 || rw.og == 7;
  constexpr int oy = rw.og == 2 || rw.og == 4 || rw.og == 6 || rw.og == 7;
  constexpr int oz = rw.og == 3 || rw.og == 5 || rw.og == 6 || rw.og == 7;
  if (i > g.nx - ox || j > g.ny - oy || k > g.nz - oz) return;
  const int64_t idx = int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy;
  float* yo = y + int64_t(rw.out) * g.arr + idx;
  const bool bnd = 2 * i + ox == 0 || 2 * i + ox == 2 * g.nx || 2 * j + oy == 0 || 2 * j + oy == 2 * g.ny ||
                   2 * k + oz == 0 || 2 * k + oz == 2 * g.nz;
  float a0, a1, a2;
  if (!bnd || rw.all) {
    a0 = tseg<PL, rw.t0, float>(tab, s, std::make_integer_sequence<int, rw.n0>{});
    a1 = tseg<PL, rw.t0 + rw.n0, float>(tab, s, std::make_integer_sequence<int, rw.n1>{});
    if (!bnd) a2 = tseg<PL, rw.t0 + rw.n0 + rw.n1, float>(tab, s, std::make_integer_sequence<int, rw.n2>{});
    else a2 = rw.n2 > 0 ? tboundary_seg2(g, op, R, i, j, k, x, idx) : 0.f;
  } else {
    if (MODE != MODE_ADD) *yo = 0.f;
    return;
  }
  float v = a0;
  if (VARNU) v += float(g.esc[k]) * a1 + float(g.eisc[k]) * a2;
  else v += a1 + a2;
  if (MODE == MODE_SET) *yo = v;
  else if (MODE == MODE_RES) *yo = b[int64_t(rw.out) * g.arr + idx] - v;
  else *yo += alpha * v;
}

// asynchronous 4-byte global -> shared copy (zero-filled when !valid; the
// source address is then not read)
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc, bool valid) {
  const unsigned saddr = static_cast<unsigned>(__cvta_generic_to_shared(sdst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(saddr), "l"(gsrc), "r"(valid ? 4 : 0)
               : "memory");
}

// copy slot `SL` (input array A) of the tile, lattice sites [i0-1, i0+TI] x
// [j0-1, j0+TJ] x [k0-1, k0+TK] (sites beyond the lattice's zero ring read
// 0): warp w copies tile rows w, w+8, ... (34 sites along i each), all copies
// in flight at once
template <int SL, int A>
__device__ __forceinline__ void load_slot(const Geo& g, const float* __restrict__ x, float* sm, int i0, int j0,
                                          int k0) {
  const float* xa = x + int64_t(A) * g.arr;
  const int lane = int(threadIdx.x) & 31, warp = int(threadIdx.x) >> 5;
  for (int row = warp; row < TY * TZ; row += kTileThreads / 32) {
    const int kk = row / TY, jj = row - kk * TY;
    const int j = j0 - 1 + jj, k = k0 - 1 + kk;
    const bool rowok = j <= g.ny + 1 && k <= g.nz + 1;
    const float* src = xa + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy + i0;   // site (i0-1, j, k)
    float* dst = sm + SL * VOL + row * TX;
    cp_async4(dst + lane, rowok ? src + lane : xa, rowok && i0 - 1 + lane <= g.nx + 1);
    if (lane < TX - 32) cp_async4(dst + 32 + lane, rowok ? src + 32 + lane : xa, rowok && i0 + 31 + lane <= g.nx + 1);
  }
}

template <class PL, int B, int... I>
__device__ __forceinline__ void load_tile(const Geo& g, const float* __restrict__ x, float* sm, int i0, int j0, int k0,
                                          std::integer_sequence<int, I...>) {
  (load_slot<I, PL::arrs[PL::blocks[B].a0 + I]>(g, x, sm, i0, j0, k0), ...);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int DISC, int VARNU, int OP, int MODE, int B, class Tab, int... I>
__device__ __forceinline__ void tile_rows_of_block(const Geo& g, int i, int j, int k, const float* s,
                                                   const float* __restrict__ x, const float* __restrict__ b,
                                                   float* __restrict__ y, float alpha, const OpDev& op, const Tab& tab,
                                                   std::integer_sequence<int, I...>) {
  using PL = gen::P<DISC, VARNU, OP>;
  (tile_row<DISC, VARNU, OP, MODE, PL::rows[PL::blocks[B].r0 + I]>(g, i, j, k, s, x, b, y, alpha, op, tab), ...);
}

template <int DISC, int VARNU, int OP, int MODE, int B>
__global__ void __launch_bounds__(kTileThreads)
    k_rows_tile(Geo g, const float* __restrict__ x, const float* __restrict__ b, float* __restrict__ y, float alpha,
                OpDev op, int nti, int ntj, const __grid_constant__ FastTab<float, gen::S<DISC, VARNU, OP>::N> tab) {
  using PL = gen::P<DISC, VARNU, OP>;
  constexpr gen::BlockT blk = PL::blocks[B];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = reinterpret_cast<float*>(smem_raw);
  const int tile = int(blockIdx.x);
  const int tk = tile / (nti * ntj), rem = tile - tk * nti * ntj, tj = rem / nti, ti = rem - tj * nti;
  const int i0 = ti * TI, j0 = tj * TJ, k0 = tk * TK;
  load_tile<PL, B>(g, x, sm, i0, j0, k0, std::make_integer_sequence<int, blk.na>{});
  __syncthreads();
  for (int q = threadIdx.x; q < TI * TJ * TK; q += kTileThreads) {
    const int kk = q / (TI * TJ), r = q - kk * TI * TJ, jj = r / TI, ii = r - jj * TI;
    const int i = i0 + ii, j = j0 + jj, k = k0 + kk;
    if (i > g.nx || j > g.ny || k > g.nz) continue;
    const float* s = sm + (ii + 1) + (jj + 1) * TX + (kk + 1) * TX * TY;
    tile_rows_of_block<DISC, VARNU, OP, MODE, B>(g, i, j, k, s, x, b, y, alpha, op, tab,
                                                 std::make_integer_sequence<int, blk.nr>{});
  }
}

template <int DISC, int VARNU, int OP, int MODE, int B>
void set_tile_attr() {
  using PL = gen::P<DISC, VARNU, OP>;
  cudaFuncSetAttribute(k_rows_tile<DISC, VARNU, OP, MODE, B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       int(PL::blocks[B].na * VOL * sizeof(float)));
}

template <int DISC, int VARNU, int OP, int MODE, int B>
void launch_block(const Geo& g, const OpDev& od, const void* tab, const float* x, const float* b, float* y, float alpha,
                  cudaStream_t s) {
  using PL = gen::P<DISC, VARNU, OP>;
  using Tab = FastTab<float, gen::S<DISC, VARNU, OP>::N>;
  if constexpr (B < PL::NB) {
    const int nti = (g.nx + 1 + TI - 1) / TI, ntj = (g.ny + 1 + TJ - 1) / TJ, ntk = (g.nz + 1 + TK - 1) / TK;
    ++g_launches;
    k_rows_tile<DISC, VARNU, OP, MODE, B><<<nti * ntj * ntk, kTileThreads, PL::blocks[B].na * VOL * sizeof(float), s>>>(
        g, x, b, y, alpha, od, nti, ntj, *static_cast<const Tab*>(tab));
    launch_block<DISC, VARNU, OP, MODE, B + 1>(g, od, tab, x, b, y, alpha, s);
  }
}

template <int DISC, int VARNU, int OP, int MODE, int B>
void init_blocks() {
  using PL = gen::P<DISC, VARNU, OP>;
  if constexpr (B < PL::NB) {
    set_tile_attr<DISC, VARNU, OP, MODE, B>();
    init_blocks<DISC, VARNU, OP, MODE, B + 1>();
  }
}

template <int DISC, int VARNU>
void init_disc() {
  init_blocks<DISC, VARNU, OP_FULL, MODE_SET, 0>();
  init_blocks<DISC, VARNU, OP_FULL, MODE_RES, 0>();
  init_blocks<DISC, VARNU, OP_BT, MODE_RES, 0>();
  init_blocks<DISC, VARNU, OP_BC, MODE_RES, 0>();
}

template <int DISC, int VARNU>
bool launch_disc(int op, int mode, const Geo& g, const OpDev& od, const void* tab, const float* x, const float* b,
                 float* y, float alpha, cudaStream_t s) {
  if (op == OP_FULL && mode == MODE_SET) launch_block<DISC, VARNU, OP_FULL, MODE_SET, 0>(g, od, tab, x, b, y, alpha, s);
  else if (op == OP_FULL && mode == MODE_RES) launch_block<DISC, VARNU, OP_FULL, MODE_RES, 0>(g, od, tab, x, b, y, alpha, s);
  else if (op == OP_BT && mode == MODE_RES) launch_block<DISC, VARNU, OP_BT, MODE_RES, 0>(g, od, tab, x, b, y, alpha, s);
  else if (op == OP_BC && mode == MODE_RES) launch_block<DISC, VARNU, OP_BC, MODE_RES, 0>(g, od, tab, x, b, y, alpha, s);
  else return false;
  return true;
}

}  // namespace

void tile_init() {
  init_disc<1, 0>();
  init_disc<1, 1>();
  init_disc<2, 0>();
  init_disc<2, 1>();
}

bool tile_rows(int disc, int varnu, int op, int mode, const Geo& g, const OpDev& od, const void* tab, const float* x,
               const float* b, float* y, double alpha, cudaStream_t s) {
  const float a = float(alpha);
  if (disc == 1 && !varnu) return launch_disc<1, 0>(op, mode, g, od, tab, x, b, y, a, s);
  if (disc == 1) return launch_disc<1, 1>(op, mode, g, od, tab, x, b, y, a, s);
  if (!varnu) return launch_disc<2, 0>(op, mode, g, od, tab, x, b, y, a, s);
  return launch_disc<2, 1>(op, mode, g, od, tab, x, b, y, a, s);
}

}  // namespace hhg
