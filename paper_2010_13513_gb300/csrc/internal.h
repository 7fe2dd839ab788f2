// Internal declarations of the HHG Stokes library (host C++ and CUDA).
//
// Data layout in HBM (one block vector of level l):
//   [u1 g0 .. u1 g(G-1) | u2 g0 .. | u3 g0 .. | p]     (3G + 1 group arrays)
// G = 1 for P1-P1 (vertex DoFs), G = 8 for P2-P1 (vertex + 7 edge groups,
// Sec. 2.2).  Every group array is box-shaped over the coarse index (i,j,k),
// 0 <= i <= nx (+1 halo layer on each side, zero), x fastest:
//   index(i,j,k) = (i+1) + (j+1) sx + (k+1) sy,
// with the j pitch sx = nx + 3, rounded up to a multiple of four on levels
// with nx >= 64 (the extra entries of a row are padding, zero).
// Group g with parity offset o_g holds the DoF at doubled position
// 2 (i,j,k) + o_g; entries past the group's extent are padding (zero).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/hhg.h"

namespace hhg {

constexpr int kMaxGroups = 8;
// parity offsets of the DoF groups, in the multicolour Gauss-Seidel order:
// vertex, x, y, z, xy, xz, yz, xyz
constexpr int kGroupOff[8][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1},
                                 {1, 1, 0}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

inline int group_of_parity(int ox, int oy, int oz) {
  for (int g = 0; g < 8; ++g)
    if (kGroupOff[g][0] == ox && kGroupOff[g][1] == oy && kGroupOff[g][2] == oz) return g;
  return -1;
}

// ------------------------------------------------------------ level geometry
struct Geo {
  int nx, ny, nz;       // cells per direction
  int sx;               // pitch of j
  int64_t sy;           // pitch of k
  int64_t arr;          // elements per group array (padded to a multiple of 64)
  int G;                // velocity groups
  double h;             // mesh width
  double nu_ah;         // nu_a * h (row scaling exp(zs * nu_ah * k))
  const double* esc;    // exp(+nu_ah k), k = 0..nz (device; set when nu_a != 0)
  const double* eisc;   // exp(-nu_ah k)
};

inline Geo make_geo(int mx, int my, int mz, int level, int G, double H, double nu_a) {
  Geo g;
  const int n = 1 << level;
  g.nx = mx * n; g.ny = my * n; g.nz = mz * n;
  // large levels: a multiple of four (16-byte aligned quads of sites for the
  // streaming kernels); small levels keep the tight pitch (their smoother
  // holds the whole level in shared memory)
  g.sx = g.nx + 3;
  if (g.nx >= 64) g.sx = (g.sx + 3) / 4 * 4;
  g.sy = int64_t(g.sx) * (g.ny + 3);
  int64_t a = g.sy * (g.nz + 3);
  g.arr = (a + 63) / 64 * 64;
  g.G = G;
  g.h = H / n;
  g.nu_ah = nu_a * g.h;
  g.esc = nullptr;
  g.eisc = nullptr;
  return g;
}

// ------------------------------------------------------- stencil row tables
// A term reads in_arr at (coarse index of the row) + (di,dj,dk).  Interior
// rows use the terms merged over all adjacent cubes; rows on the domain
// boundary use the per-cube terms and keep a term only if its cube
// (row index + (cx,cy,cz)) lies inside the domain.
struct HTerm {
  int in_arr;
  int di, dj, dk;
  int cx, cy, cz;       // cube offset (per-cube terms only)
  double w;
};

// A row has three term segments by viscosity scaling: seg[0] unscaled,
// seg[1] times exp(+nu_a h k) (A), seg[2] times exp(-nu_a h k) (C, PSPG load,
// lumped 1/nu mass), k the row's coarse z index.
struct HRow {
  int out_arr;
  int og;               // group of the row DoF
  bool all_rows;        // false: velocity Dirichlet rows are written as 0
  std::vector<HTerm> seg[3];    // merged terms; in an A row seg[1] starts with the diagonal
  std::vector<HTerm> bseg[3];   // per-cube terms
};

struct HOperator {
  std::vector<HRow> rows;
};

// device-side forms
struct DTerm {
  int arr;
  int off;              // linear offset di + dj sx + dk sy
};
struct DTermB {
  int arr;
  int off;
  int cx, cy, cz, pad;
};
struct DRow {
  int out_arr, og, all_rows, pad;
  int t0, n0, n1, n2;       // interior terms: [t0, t0+n0) seg 0, then n1 of seg 1, n2 of seg 2
  int b0, m0, m1, m2;       // per-cube terms, same segment order
};

struct OpDev {
  const DRow* rows;
  int nrows;
  const DTerm* terms;
  const double* w64;
  const float* w32;
  const DTermB* bterms;
  const double* bw64;
  const float* bw32;
};

// ------------------------------------------------------- transfer tables
// Prolongation I_{l-1}^l: a fine DoF at doubled fine position P (units h_f/2)
// has class kappa = P mod 4 (P2) or (P/2) mod 2 (P1) and reads coarse DoFs
// (g_c, a + d) with a = P >> 2 (P2) or (P/2) >> 1 (P1).
// Restriction (transpose): a coarse DoF (g_c, a) reads fine DoFs
// (g_f, 2a + e).
struct HXTerm {
  int arr;              // coarse group (prolongation) or fine group (restriction)
  int di, dj, dk;
  double w;
};
struct HTransfer {
  int order;                                 // 1 or 2
  int nclass;                                // 8 (P1) or 64 (P2)
  std::vector<std::vector<HXTerm>> prol;     // [nclass]
  std::vector<std::vector<HXTerm>> restr;    // [groups]
};
struct DXTerm {
  int arr, di, dj, dk;
};
struct XferDev {
  int order, nclass, ngroups;
  int rmax;                   // most restriction terms of a group
  const int* pcls_start;      // nclass + 1
  const DXTerm* pterms;
  const double* pw64;
  const float* pw32;
  const int* rg_start;        // ngroups + 1
  const DXTerm* rterms;
  const double* rw64;
  const float* rw32;
};

// ------------------------------------------------------------ host builders
enum OpId {
  OP_FULL = 0, OP_A, OP_BT, OP_B, OP_C, OP_MASS, OP_BC, OP_MVINT, OP_LOAD, OP_MLHAT, OP_ML, OP_COUNT
};

// element-level quantities of the 6 Kuhn classes and the stencil builder
struct StencilSet {
  HOperator op[OP_COUNT];
  std::vector<double> diagA;      // per group: diagonal of A (relative weights)
};
StencilSet build_stencils(int disc, double h, double nu_a, bool pspg_rhs);
HTransfer build_transfer(int order);

// ------------------------------------------------------------ device launch
struct Launch;  // fwd

}  // namespace hhg
