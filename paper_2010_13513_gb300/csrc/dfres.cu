// Refinement residual of the mixed-precision solve in double-float arithmetic.
//
// The mixed solve (FP32 V-cycles inside an FP64 iterative refinement) needs
// the outer residual r = b - calA x of every FMG stage to well below FP32
// rounding.  FP64 arithmetic gives that, but on this GPU FP64 FMAs run at
// about 1/54 of the FP32 rate (1.26 against 68.5 TFLOP/s measured), so the
// FP64 residual of the finest level is bound by them (it was the largest
// single kernel of the level-7 solve).  Here
// every FP64 value v is carried as two FP32 numbers v = v_hi + v_lo (47
// significant bits, split by integer bit operations, no FP64 instruction on
// the common path), and each row is evaluated as the compensated dot product
// "Dot2" of Ogita, Rump and Oishi (Accurate sum and dot product, SIAM J. Sci.
// Comput. 26(6), 2005): the product w_hi x_hi is split exactly into p + e by
// one FMA, p enters the running sum through Knuth's error-free TwoSum (The Art
// of Computer Programming, vol. 2, Sec. 4.2.2), and the sum's rounding errors,
// e and the small products w_lo x_hi + w_hi x_lo are collected in a second
// FP32 accumulator.  With u = 2^-24 and n terms the computed row differs from
// the exact one by at most about u |r| + (n^2 u^2 + 2^-46) sum_j |a_ij x_j|: as
// if evaluated in 47-bit arithmetic and then rounded to FP32, the precision
// the V-cycle takes its right-hand side in.
//
// Work layout (as the vector row kernels of the FP32/FP64 path): grid x over
// the padded (i, j) plane in warps of 4 x 32 positions, y over groups of kp
// planes, z over the rows of the operator; on large levels a thread
// evaluates 4 sites 32 positions apart (two at a time with the paired FP32
// f32x2 instructions) on 2 planes, on small ones 1 site on 1 plane.
// The terms of a row are a loop over weights and offsets in the constant
// bank, so a row's code stays small in the instruction cache.
// Boundary pressure rows (P1-P1: the C terms of the cubes inside the box) add
// their per-cube C terms in FP64; they are a few per cent of the pressure
// rows.  With a variable viscosity nu = exp(a z) the segments of a row are
// summed apart and scaled by the row's FP64 factors exp(+-a h k) in
// double-float arithmetic.
#include "dfres.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "batch.h"
#include "kernels.h"
#include "structure.inc"

namespace hhg {
namespace {

template <int N>
struct DfTab {
  float wh[N];       // weights: w = wh + wl (|w - wh - wl| <= 2^-48 |w|)
  float wl[N];
  int off[N];        // linear offsets arr * array_stride + di + dj sx + dk sy
};

template <int DISC, int VARNU>
using DfTabOf = DfTab<gen::S<DISC, VARNU, OP_FULL>::N>;

// v = hi + lo with |v - hi - lo| < 2^-46 |v|: hi takes the leading 24 bits of
// v's significand, lo the next 23 (both truncated).  For v = 0, |v| < 2^-100
// or |v| >= 2^126, hi = fl32(v) and lo = 0 (an FP64 conversion off the common
// path).
__device__ __forceinline__ void split_df(double v, float& hi, float& lo) {
  const unsigned long long u = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned top = unsigned(u >> 32);
  const unsigned sgn = top & 0x80000000u;
  const int e = int((top >> 20) & 0x7ffu);           // biased FP64 exponent
  if (e >= 923 && e <= 1148) {
    // FP32 exponent field e - 1023 + 127; significand bits 51..29
    hi = __uint_as_float(sgn | (unsigned(e - 896) << 23) | unsigned((u >> 29) & 0x7fffffu));
    // bits 28..6 of the significand scaled by 2^(e - 1069): (1 + f) 2^E - 2^E
    // with E = e - 1046, an exact FP32 subtraction
    const unsigned eb = unsigned(e - 919) << 23;
    lo = __fsub_rn(__uint_as_float(sgn | eb | (unsigned(u & 0x1fffffffu) >> 6)), __uint_as_float(sgn | eb));
  } else if (e == 0) {
    hi = __uint_as_float(sgn);                       // +-0 (and FP64 subnormals, < 2^-1022)
    lo = 0.0f;
  } else {
    hi = __double2float_rn(v);
    lo = 0.0f;
  }
}

// one Dot2 step: (s, c) += (wh + wl) (xh + xl); the rounded operations are
// the _rn intrinsics, which the compiler never contracts into FMAs
__device__ __forceinline__ void dot2_term(float wh, float wl, float xh, float xl, float& s, float& c) {
  const float p = __fmul_rn(wh, xh);
  float e = __fmaf_rn(wh, xh, -p);                   // wh xh = p + e exactly
  e = __fmaf_rn(wl, xh, e);
  e = __fmaf_rn(wh, xl, e);
  const float t = __fadd_rn(s, p);                   // TwoSum: s + p = t + d exactly
  const float z = __fsub_rn(t, s);
  const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(d, e));
}

// a - b on both halves (sub.rn.f32x2: each half rounds as the scalar
// subtraction)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rr;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rr, ra, rb;\n mov.b64 {%0, %1}, rr;\n}"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// dot2_term on two sites at once with the paired FP32 instructions (each
// half of an f32x2 operation rounds as the scalar one, so the sums are those
// of dot2_term bit for bit)
__device__ __forceinline__ void dot2_term2(float2 wh, float2 wl, float2 xh, float2 xl, float2& s, float2& c) {
  const float2 p = __fmul2_rn(wh, xh);
  float2 e = __ffma2_rn(wh, xh, make_float2(-p.x, -p.y));
  e = __ffma2_rn(wl, xh, e);
  e = __ffma2_rn(wh, xl, e);
  const float2 t = __fadd2_rn(s, p);
  const float2 z = sub2(t, s);
  const float2 d = __fadd2_rn(sub2(s, sub2(t, z)), sub2(p, z));
  s = t;
  c = __fadd2_rn(c, __fadd2_rn(d, e));
}

// terms [T0, T0 + N) of a row at NS sites 32 positions apart (idx + 32 v);
// an even NS runs the sites in pairs
template <int T0, int N, int NS, class Tab>
__device__ __forceinline__ void dot2_seg(const Tab& tab, const float* __restrict__ xh, const float* __restrict__ xl,
                                         int64_t idx, float (&s)[NS], float (&c)[NS]) {
  if constexpr (NS % 2 == 0) {
    float2 s2[NS / 2], c2[NS / 2];
#pragma unroll
    for (int h = 0; h < NS / 2; ++h) {
      s2[h] = make_float2(s[2 * h], s[2 * h + 1]);
      c2[h] = make_float2(c[2 * h], c[2 * h + 1]);
    }
#pragma unroll 4
    for (int t = T0; t < T0 + N; ++t) {
      const float wh = tab.wh[t], wl = tab.wl[t];
      const int64_t q = idx + tab.off[t];
#pragma unroll
      for (int h = 0; h < NS / 2; ++h)
        dot2_term2(make_float2(wh, wh), make_float2(wl, wl),
                   make_float2(__ldg(xh + q + 64 * h), __ldg(xh + q + 64 * h + 32)),
                   make_float2(__ldg(xl + q + 64 * h), __ldg(xl + q + 64 * h + 32)), s2[h], c2[h]);
    }
#pragma unroll
    for (int h = 0; h < NS / 2; ++h) {
      s[2 * h] = s2[h].x; s[2 * h + 1] = s2[h].y;
      c[2 * h] = c2[h].x; c[2 * h + 1] = c2[h].y;
    }
  } else {
#pragma unroll 4
    for (int t = T0; t < T0 + N; ++t) {
      const float wh = tab.wh[t], wl = tab.wl[t];
      const int64_t q = idx + tab.off[t];
#pragma unroll
      for (int v = 0; v < NS; ++v) dot2_term(wh, wl, __ldg(xh + q + 32 * v), __ldg(xl + q + 32 * v), s[v], c[v]);
    }
  }
}

// per-cube C terms of boundary pressure row r at site (i, j, k) (index idx),
// the cubes inside the box only, in FP64 with x = xh + xl
__device__ double boundary_c64(const Geo& g, const OpDev& op, int r, int i, int j, int k, const float* xh,
                               const float* xl, int64_t idx) {
  const DRow row = op.rows[r];
  double a = 0.0;
  for (int t = row.b0 + row.m0 + row.m1; t < row.b0 + row.m0 + row.m1 + row.m2; ++t) {
    const DTermB tm = op.bterms[t];
    const int qx = i + tm.cx, qy = j + tm.cy, qz = k + tm.cz;
    if (qx < 0 || qy < 0 || qz < 0 || qx >= g.nx || qy >= g.ny || qz >= g.nz) continue;
    const int64_t q = int64_t(tm.arr) * g.arr + idx + tm.off;
    a += __ldg(op.bw64 + t) * (double(__ldg(xh + q)) + double(__ldg(xl + q)));
  }
  return a;
}

// (s, c) += a (u + v) for an FP64 factor a = ah + al: ah u = p + e exactly
// (FMA), the small products into e, p into the sum by TwoSum
__device__ __forceinline__ void df_add_scaled(double a, float u, float v, float& s, float& c) {
  float ah, al;
  split_df(a, ah, al);
  const float p = __fmul_rn(ah, u);
  float e = __fmaf_rn(ah, u, -p);
  e = __fmaf_rn(ah, v, e);
  e = __fmaf_rn(al, u, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  s = t;
  c = __fadd_rn(c, __fadd_rn(d, e));
}

// the residual of row R at one site from its sums: (s, c) over segment 0
// (and segment 1 with a constant viscosity), (s1, c1) over segment 1 with a
// variable one (scaled by exp(+nu_a h k)), (s2, c2) over segment 2 (C; scaled
// by exp(-nu_a h k) with a variable viscosity); bnd: the site lies on the box
// boundary
template <int OUT, int ALL, int N2, int VARNU>
__device__ __forceinline__ void df_store(const Geo& g, const OpDev& op, int R, int i, int j, int k, bool bnd,
                                         const float* xh, const float* xl, int64_t idx, float s, float c, float s1,
                                         float c1, float s2, float c2, const double* __restrict__ b,
                                         float* __restrict__ r) {
  const int64_t iy = int64_t(OUT) * g.arr + idx;
  if (bnd && !ALL) {                                 // Dirichlet velocity row
    r[iy] = 0.0f;
    return;
  }
  const double bv = __ldg(b + iy);
  const double es = VARNU ? __ldg(g.esc + k) : 1.0, eis = VARNU ? __ldg(g.eisc + k) : 1.0;
  if (N2 > 0 && bnd) {
    // boundary pressure row: the clipped C terms in FP64
    const double cb = boundary_c64(g, op, R, i, j, k, xh, xl, idx);
    const double a1 = VARNU ? es * (double(s1) + double(c1)) : 0.0;
    r[iy] = __double2float_rn(bv - (double(s) + double(c)) - a1 - eis * cb);
    return;
  }
  if (VARNU) {
    df_add_scaled(es, s1, c1, s, c);
    if (N2 > 0) df_add_scaled(eis, s2, c2, s, c);
  } else if (N2 > 0) {                               // (s, c) += (s2, c2)
    const float t = __fadd_rn(s, s2);
    const float z = __fsub_rn(t, s);
    const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(s2, z));
    s = t;
    c = __fadd_rn(c, __fadd_rn(c2, d));
  }
  float bh, bl;
  split_df(bv, bh, bl);
  // (bh + bl) - (s + c): TwoSum of bh and -s, then the small parts
  const float t = __fsub_rn(bh, s);
  const float z = __fsub_rn(t, bh);
  const float d = __fadd_rn(__fsub_rn(bh, __fsub_rn(t, z)), __fsub_rn(-s, z));
  r[iy] = __fadd_rn(t, __fsub_rn(__fadd_rn(d, bl), c));
}

// row R = (OUT, OG, ALL, T0, N0, N1, N2) on the sites of the block: the
// indexing of the vector row kernels (four runs of 32 positions per warp; a
// warp whose last run passes the group's last site takes its sites one by one)
template <int V, int VARNU, int OUT, int OG, int ALL, int T0, int N0, int N1, int N2, class Tab>
__device__ __forceinline__ void df_rows(const uint3 bid, const Geo& g, int R, const float* __restrict__ xh,
                                        const float* __restrict__ xl, const double* __restrict__ b,
                                        float* __restrict__ r, const OpDev& op, const Tab& tab, int kp) {
  constexpr int ox = OG == 1 || OG == 4 || OG == 5 || OG == 7;
  constexpr int oy = OG == 2 || OG == 4 || OG == 6 || OG == 7;
  constexpr int oz = OG == 3 || OG == 5 || OG == 6 || OG == 7;
  const int m0 = ((bid.x * blockDim.x + threadIdx.x) >> 5) * (32 * V);
  const int lane = int(threadIdx.x & 31);
  const int mlast = (g.ny - oy) * g.sx + (g.nx - ox);
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
        const bool bnd = 2 * i + ox == 0 || 2 * i + ox == 2 * g.nx || 2 * j + oy == 0 || 2 * j + oy == 2 * g.ny ||
                         2 * k + oz == 0 || 2 * k + oz == 2 * g.nz;
        const int64_t idx = int64_t(m) + 1 + g.sx + int64_t(k + 1) * g.sy;
        float s[1] = {0.0f}, c[1] = {0.0f}, s1[1] = {0.0f}, c1[1] = {0.0f}, s2[1] = {0.0f}, c2[1] = {0.0f};
        if (!bnd || ALL) {
          if (VARNU) {
            dot2_seg<T0, N0, 1>(tab, xh, xl, idx, s, c);
            dot2_seg<T0 + N0, N1, 1>(tab, xh, xl, idx, s1, c1);
          } else {
            dot2_seg<T0, N0 + N1, 1>(tab, xh, xl, idx, s, c);
          }
          if (N2 > 0 && !bnd) dot2_seg<T0 + N0 + N1, N2, 1>(tab, xh, xl, idx, s2, c2);
        }
        df_store<OUT, ALL, N2, VARNU>(g, op, R, i, j, k, bnd, xh, xl, idx, s[0], c[0], s1[0], c1[0], s2[0], c2[0], b,
                                      r);
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
    float s[V], c[V], s1[V], c1[V], s2[V], c2[V];
#pragma unroll
    for (int v = 0; v < V; ++v) s[v] = c[v] = s1[v] = c1[v] = s2[v] = c2[v] = 0.0f;
    if (VARNU) {
      dot2_seg<T0, N0, V>(tab, xh, xl, idx, s, c);
      dot2_seg<T0 + N0, N1, V>(tab, xh, xl, idx, s1, c1);
    } else {
      dot2_seg<T0, N0 + N1, V>(tab, xh, xl, idx, s, c);
    }
    if (N2 > 0) dot2_seg<T0 + N0 + N1, N2, V>(tab, xh, xl, idx, s2, c2);
    const bool bk = 2 * k + oz == 0 || 2 * k + oz == 2 * g.nz;
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (okv[v])
        df_store<OUT, ALL, N2, VARNU>(g, op, R, iv[v], jv[v], k, bijv[v] || bk, xh, xl, idx + 32 * v, s[v], c[v],
                                      s1[v], c1[v], s2[v], c2[v], b, r);
  }
}

template <class S, int R, class F>
__device__ __forceinline__ void by_row(int r, F&& f) {
  if constexpr (R < S::R) {
    if (r == R) f(std::integral_constant<int, R>{});
    else by_row<S, R + 1>(r, f);
  }
}

template <int DISC, int VARNU, int V, class Tab>
__device__ __forceinline__ void res_df_body(const uint3 bid, const Geo& g, const float* __restrict__ xh,
                                            const float* __restrict__ xl, const double* __restrict__ b,
                                            float* __restrict__ r, const OpDev& op, int kp, const Tab& tab) {
  using S = gen::S<DISC, VARNU, OP_FULL>;
  by_row<S, 0>(int(bid.z), [&](auto rc) {
    constexpr int R = decltype(rc)::value;
    constexpr gen::RowS rw = S::rows[R];
    df_rows<V, VARNU, rw.out, rw.og, rw.all, rw.t0, rw.n0, rw.n1, rw.n2>(bid, g, R, xh, xl, b, r, op, tab, kp);
  });
}

template <int DISC, int VARNU, int V>
__global__ void __launch_bounds__(128) k_res_df(Geo g, const float* __restrict__ xh, const float* __restrict__ xl,
                                                const double* __restrict__ b, float* __restrict__ r, OpDev op, int kp,
                                                const __grid_constant__ DfTabOf<DISC, VARNU> tab) {
  res_df_body<DISC, VARNU, V>(blockIdx, g, xh, xl, b, r, op, kp, tab);
}

// hi[q] + lo[q] = x[q] (split_df), two elements per thread and step (n even)
__device__ __forceinline__ void split_df_body(const uint3 bid, const uint3 gd, const double2* __restrict__ x,
                                              float2* __restrict__ hi, float2* __restrict__ lo, int64_t n2) {
  for (int64_t q = bid.x * int64_t(blockDim.x) + threadIdx.x; q < n2; q += int64_t(gd.x) * blockDim.x) {
    const double2 v = x[q];
    float2 h, l;
    split_df(v.x, h.x, l.x);
    split_df(v.y, h.y, l.y);
    hi[q] = h;
    lo[q] = l;
  }
}

__global__ void k_split_df(const double2* __restrict__ x, float2* __restrict__ hi, float2* __restrict__ lo,
                           int64_t n2) {
  split_df_body(blockIdx, gridDim, x, hi, lo, n2);
}

// the same two kernels as work items of a merged batch launch (batch.h; the
// weight table as a device copy)
struct SplitA { const double2* x; float2* hi; float2* lo; int64_t n2; };
template <class Tab>
struct ResDfA { Geo g; const float* xh; const float* xl; const double* b; float* r; OpDev op; int kp; const Tab* tab; };

__global__ void kb_split_df(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<SplitA>(items, n, bid, gd);
  split_df_body(bid, gd, it.a.x, it.a.hi, it.a.lo, it.a.n2);
}

template <int DISC, int VARNU, int V>
__global__ void __launch_bounds__(128) kb_res_df(const void* items, int n) {
  uint3 bid, gd;
  const auto& it = batch_item<ResDfA<DfTabOf<DISC, VARNU>>>(items, n, bid, gd);
  const auto& a = it.a;
  res_df_body<DISC, VARNU, V>(bid, a.g, a.xh, a.xl, a.b, a.r, a.op, a.kp, *a.tab);
}

constexpr int kDfThreads = 128;
// levels with at most this many lattice sites take one site and one plane
// per thread (the row loops are latency-bound; more threads hide it), larger
// ones four sites and two planes
constexpr int64_t kDfSmallSites = 300000;

template <int DISC, int VARNU>
void launch_df(const Geo& g, const OpDev& od, const char* tab, const double* x, const double* b, float* xh, float* xl,
               float* r, cudaStream_t s) {
  using S = gen::S<DISC, VARNU, OP_FULL>;
  using Tab = DfTabOf<DISC, VARNU>;
  const int64_t n = (3 * int64_t(g.G) + 1) * g.arr;  // a multiple of 64
  const int64_t n2 = n / 2;
  const dim3 sgrd(unsigned(std::min<int64_t>((n2 + 255) / 256, 152 * 8)));
  const SplitA sa{reinterpret_cast<const double2*>(x), reinterpret_cast<float2*>(xh), reinterpret_cast<float2*>(xl),
                  n2};
  const bool small = int64_t(g.nx + 1) * (g.ny + 1) * (g.nz + 1) <= kDfSmallSites;
  const int v = small ? 1 : 4, kp = small ? 1 : 2;
  // warps of v x 32 positions over the padded plane up to the last site
  const int64_t warps = ((int64_t(g.ny) * g.sx + g.nx + 1) + 32 * v - 1) / (32 * v);
  const dim3 grd(unsigned((warps * 32 + kDfThreads - 1) / kDfThreads), unsigned((g.nz + 1 + kp - 1) / kp),
                 unsigned(S::R));
  if (g_rec) {                                       // a batch records: two work items
    const Tab* dt = static_cast<const Tab*>(g_rec->table(tab, sizeof(Tab)));
    g_rec->add(reinterpret_cast<const void*>(kb_split_df), sgrd, dim3(256), 0, 1, sa);
    g_rec->add(small ? reinterpret_cast<const void*>(kb_res_df<DISC, VARNU, 1>)
                     : reinterpret_cast<const void*>(kb_res_df<DISC, VARNU, 4>),
               grd, dim3(kDfThreads), 0, 1, ResDfA<Tab>{g, xh, xl, b, r, od, kp, dt});
    return;
  }
  Tab tb;
  std::memcpy(&tb, tab, sizeof(tb));
  ++g_launches;
  k_split_df<<<sgrd, 256, 0, s>>>(sa.x, sa.hi, sa.lo, n2);
  ++g_launches;
  if (small) k_res_df<DISC, VARNU, 1><<<grd, kDfThreads, 0, s>>>(g, xh, xl, b, r, od, kp, tb);
  else k_res_df<DISC, VARNU, 4><<<grd, kDfThreads, 0, s>>>(g, xh, xl, b, r, od, kp, tb);
}

void df_launch(int disc, int varnu, const Geo& g, const OpDev& od, const char* tab, const double* x, const double* b,
               float* xh, float* xl, float* r, cudaStream_t s) {
  if (disc == 1 && !varnu) launch_df<1, 0>(g, od, tab, x, b, xh, xl, r, s);
  else if (disc == 1) launch_df<1, 1>(g, od, tab, x, b, xh, xl, r, s);
  else if (!varnu) launch_df<2, 0>(g, od, tab, x, b, xh, xl, r, s);
  else launch_df<2, 1>(g, od, tab, x, b, xh, xl, r, s);
}

}  // namespace

bool df_supported(int disc, int varnu) { return (varnu == 0 || varnu == 1) && (disc == 1 || disc == 2); }

bool df_table(int disc, int varnu, const std::vector<char>& ftab64, std::vector<char>& out) {
  out.clear();
  if (!df_supported(disc, varnu)) return false;
  const int N = disc == 1 ? (varnu ? gen::S<1, 1, OP_FULL>::N : gen::S<1, 0, OP_FULL>::N)
                          : (varnu ? gen::S<2, 1, OP_FULL>::N : gen::S<2, 0, OP_FULL>::N);
  const size_t bytes = disc == 1 ? (varnu ? sizeof(DfTabOf<1, 1>) : sizeof(DfTabOf<1, 0>))
                                 : (varnu ? sizeof(DfTabOf<2, 1>) : sizeof(DfTabOf<2, 0>));
  if (ftab64.size() < size_t(N) * 12) return false;
  // the FP64 table image: N weights, then N offsets
  const double* w = reinterpret_cast<const double*>(ftab64.data());
  const int* off = reinterpret_cast<const int*>(ftab64.data() + size_t(N) * 8);
  out.assign(bytes, 0);
  float* wh = reinterpret_cast<float*>(out.data());
  float* wl = wh + N;
  int* o = reinterpret_cast<int*>(out.data() + size_t(2 * N) * 4);
  for (int t = 0; t < N; ++t) {
    wh[t] = float(w[t]);
    wl[t] = float(w[t] - double(wh[t]));
    o[t] = off[t];
  }
  return true;
}

void df_residual(int disc, int varnu, const Geo& g, const OpDev& od, const std::vector<char>& dftab, const double* x,
                 const double* b, float* xh, float* xl, float* r, cudaStream_t s) {
  df_launch(disc, varnu, g, od, dftab.data(), x, b, xh, xl, r, s);
}

}  // namespace hhg
