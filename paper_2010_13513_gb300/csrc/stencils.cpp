// Constant per-macro stencils of the Stokes blocks on the Kuhn lattice and
// the transfer tables (host side).
//
// Sec. 2.1: after uniform refinement every micro tetrahedron is a translate
// of one of six classes, so the stencil at every interior DoF of a group is
// the same (Sec. 2.2, Table 2: eight stencils for P2, one for P1).  The
// stencil of a row is the sum of the element matrices of the micro
// tetrahedra around the row DoF.  Element matrices are integrated with a
// collapsed-coordinate Gauss-Legendre product rule (4^3 points, exact for
// the degree <= 4 integrands of P2 mass, stiffness and divergence).
//
// Variable viscosity nu = exp(a z) evaluated at the centroid of each micro
// tetrahedron: the centroid height of class s in cube q is
// h (q_z + (3 - t_s) / 4), t_s the position of the z-step in the Kuhn path, so
// nu_T = exp(a h k) * exp(a h (c_z + (3 - t_s)/4)) for a row at height k and
// cube offset c: the first factor scales the whole row (applied in the
// kernels), the second is folded into the stencil weights.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>

#include "internal.h"

namespace hhg {
namespace {

constexpr int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
constexpr int kEdge[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
constexpr double kDelta = 1.0 / 12.0;   // PSPG delta_T (Sec. 2, Eq. pspg)

struct Tet {
  int v[4][3];          // lattice coordinates (cube at origin)
  int zpos;             // position of the z step in the path
};

Tet kuhn_tet(int s) {
  Tet t{};
  int cur[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d) t.v[0][d] = 0;
  for (int step = 0; step < 3; ++step) {
    cur[kPerm[s][step]] += 1;
    for (int d = 0; d < 3; ++d) t.v[step + 1][d] = cur[d];
    if (kPerm[s][step] == 2) t.zpos = step;
  }
  return t;
}

// local DoF positions in doubled lattice units (relative to the cube origin)
void local_positions(const Tet& t, int order, std::vector<std::array<int, 3>>& pos) {
  pos.clear();
  for (int a = 0; a < 4; ++a) pos.push_back({2 * t.v[a][0], 2 * t.v[a][1], 2 * t.v[a][2]});
  if (order == 2)
    for (auto& e : kEdge)
      pos.push_back({t.v[e[0]][0] + t.v[e[1]][0], t.v[e[0]][1] + t.v[e[1]][1], t.v[e[0]][2] + t.v[e[1]][2]});
}

// -------------------------------------------------------------- quadrature
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      double dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) { double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    double dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);      // = 0.5 * 2/((1-z^2) P'^2)
  }
}

struct QuadRule {
  std::vector<std::array<double, 4>> lam;   // barycentric coordinates
  std::vector<double> w;                    // weights, sum = 1 (times |T| later)
};

QuadRule tet_rule() {
  std::vector<double> x, w;
  gauss_legendre01(4, x, w);
  QuadRule q;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 4; ++c) {
        double r1 = x[a], r2 = (1 - x[a]) * x[b], r3 = (1 - x[a]) * (1 - x[b]) * x[c];
        q.lam.push_back({1 - r1 - r2 - r3, r1, r2, r3});
        q.w.push_back(6.0 * w[a] * w[b] * w[c] * (1 - x[a]) * (1 - x[a]) * (1 - x[b]));
      }
  return q;
}

// basis values and d/d lambda_i derivatives at one point
void basis(int order, const std::array<double, 4>& l, std::vector<double>& phi,
           std::vector<std::array<double, 4>>& dphi) {
  if (order == 1) {
    phi.assign(4, 0.0);
    dphi.assign(4, {0, 0, 0, 0});
    for (int a = 0; a < 4; ++a) { phi[a] = l[a]; dphi[a][a] = 1.0; }
    return;
  }
  phi.assign(10, 0.0);
  dphi.assign(10, {0, 0, 0, 0});
  for (int a = 0; a < 4; ++a) { phi[a] = l[a] * (2 * l[a] - 1); dphi[a][a] = 4 * l[a] - 1; }
  for (int e = 0; e < 6; ++e) {
    int i = kEdge[e][0], j = kEdge[e][1];
    phi[4 + e] = 4 * l[i] * l[j];
    dphi[4 + e][i] = 4 * l[j];
    dphi[4 + e][j] = 4 * l[i];
  }
}

struct ElemMats {
  int nv;                                   // velocity local DoFs
  std::vector<double> K, Mv;                // nv x nv
  std::vector<double> D[3];                 // 4 x nv, D[d][k][j] = -int psi_k d_d phi_j
  std::vector<double> L[3];                 // 4 x nv, PSPG load
  std::vector<double> Cq, Mq;               // 4 x 4
};

ElemMats element_matrices(const Tet& t, int order, double h) {
  // geometry
  double X[4][3];
  for (int a = 0; a < 4; ++a)
    for (int d = 0; d < 3; ++d) X[a][d] = h * t.v[a][d];
  double J[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) J[r][c] = X[c + 1][r] - X[0][r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  const double vol = std::fabs(det) / 6.0;
  double gl[4][3];                        // grad lambda_a
  for (int d = 0; d < 3; ++d) {
    gl[1][d] = inv[0][d]; gl[2][d] = inv[1][d]; gl[3][d] = inv[2][d];
    gl[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
  }
  ElemMats E;
  E.nv = order == 1 ? 4 : 10;
  const int nv = E.nv;
  E.K.assign(nv * nv, 0.0); E.Mv.assign(nv * nv, 0.0);
  for (int d = 0; d < 3; ++d) { E.D[d].assign(4 * nv, 0.0); E.L[d].assign(4 * nv, 0.0); }
  E.Cq.assign(16, 0.0); E.Mq.assign(16, 0.0);

  static const QuadRule Q = tet_rule();
  std::vector<double> phi, phi1;
  std::vector<std::array<double, 4>> dphi, dphi1;
  std::vector<double> intphi(nv, 0.0);
  for (size_t q = 0; q < Q.w.size(); ++q) {
    const double wq = Q.w[q] * vol;
    basis(order, Q.lam[q], phi, dphi);
    basis(1, Q.lam[q], phi1, dphi1);
    // physical gradients
    std::vector<std::array<double, 3>> g(nv, {0, 0, 0});
    for (int a = 0; a < nv; ++a)
      for (int i = 0; i < 4; ++i)
        for (int d = 0; d < 3; ++d) g[a][d] += dphi[a][i] * gl[i][d];
    for (int a = 0; a < nv; ++a) {
      intphi[a] += wq * phi[a];
      for (int b = 0; b < nv; ++b) {
        E.K[a * nv + b] += wq * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
        E.Mv[a * nv + b] += wq * phi[a] * phi[b];
      }
    }
    for (int k = 0; k < 4; ++k) {
      for (int j = 0; j < nv; ++j)
        for (int d = 0; d < 3; ++d) E.D[d][k * nv + j] -= wq * phi1[k] * g[j][d];
      for (int l = 0; l < 4; ++l) E.Mq[k * 4 + l] += wq * phi1[k] * phi1[l];
    }
  }
  const double hT2 = std::pow(vol, 2.0 / 3.0);
  for (int k = 0; k < 4; ++k) {
    for (int l = 0; l < 4; ++l)
      E.Cq[k * 4 + l] = kDelta * hT2 * vol * (gl[k][0] * gl[l][0] + gl[k][1] * gl[l][1] + gl[k][2] * gl[l][2]);
    for (int j = 0; j < nv; ++j)
      for (int d = 0; d < 3; ++d) E.L[d][k * nv + j] = -kDelta * hT2 * gl[k][d] * intphi[j];
  }
  return E;
}

// ------------------------------------------------------------ row assembly
struct BlockAcc {
  // merged: (arr, di, dj, dk) -> w ; per cube: (arr, di, dj, dk, cx, cy, cz) -> w
  std::map<std::tuple<int, int, int, int>, double> merged;
  std::map<std::tuple<int, int, int, int, int, int, int>, double> cube;
};

// Adds the stencil of one block (element matrix family E[s], out-local x
// in-local) for the row DoF of group og of an `out_order` space.
template <class Getter>
void accumulate_block(BlockAcc& acc, int out_order, int og, int in_order, int in_arr_base, int zs, double nu_ah,
                      double coef, Getter elem) {
  const int b0[3] = {2, 2, 2};
  const int P0[3] = {2 * b0[0] + kGroupOff[og][0], 2 * b0[1] + kGroupOff[og][1], 2 * b0[2] + kGroupOff[og][2]};
  std::vector<std::array<int, 3>> pos_out, pos_in;
  for (int qz = 0; qz < 4; ++qz)
    for (int qy = 0; qy < 4; ++qy)
      for (int qx = 0; qx < 4; ++qx)
        for (int s = 0; s < 6; ++s) {
          Tet t = kuhn_tet(s);
          local_positions(t, out_order, pos_out);
          local_positions(t, in_order, pos_in);
          int a = -1;
          for (size_t m = 0; m < pos_out.size(); ++m)
            if (2 * qx + pos_out[m][0] == P0[0] && 2 * qy + pos_out[m][1] == P0[1] && 2 * qz + pos_out[m][2] == P0[2])
              a = int(m);
          if (a < 0) continue;
          const double nufac = zs == 0 ? 1.0 : std::exp(zs * nu_ah * ((qz - b0[2]) + (3 - t.zpos) / 4.0));
          for (size_t b = 0; b < pos_in.size(); ++b) {
            int P[3] = {2 * qx + pos_in[b][0], 2 * qy + pos_in[b][1], 2 * qz + pos_in[b][2]};
            int o[3] = {P[0] & 1, P[1] & 1, P[2] & 1};
            int g = group_of_parity(o[0], o[1], o[2]);
            int d[3] = {(P[0] - o[0]) / 2 - b0[0], (P[1] - o[1]) / 2 - b0[1], (P[2] - o[2]) / 2 - b0[2]};
            double w = coef * elem(s, a, int(b)) * nufac;
            acc.merged[{in_arr_base + g, d[0], d[1], d[2]}] += w;
            acc.cube[{in_arr_base + g, d[0], d[1], d[2], qx - b0[0], qy - b0[1], qz - b0[2]}] += w;
          }
        }
}

// Terms that cancel exactly for a constant viscosity (e.g. the diagonal
// directions of the P1 Laplacian) are dropped; with a variable viscosity every
// structural term is kept, so the term list never depends on the values.
bool g_drop_zeros = true;

void flush_block(const BlockAcc& acc, HRow& row, int seg, bool self_first, int self_arr, bool with_boundary) {
  double mx = 0.0;
  for (auto& kv : acc.merged) mx = std::max(mx, std::fabs(kv.second));
  double mxc = 0.0;
  for (auto& kv : acc.cube) mxc = std::max(mxc, std::fabs(kv.second));
  std::vector<HTerm> terms;
  for (auto& kv : acc.merged) {
    if (g_drop_zeros && std::fabs(kv.second) <= 1e-12 * mx) continue;
    HTerm t{std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first), 0, 0, 0,
            kv.second};
    terms.push_back(t);
  }
  if (self_first) {
    auto it = std::find_if(terms.begin(), terms.end(),
                           [&](const HTerm& t) { return t.in_arr == self_arr && !t.di && !t.dj && !t.dk; });
    if (it != terms.end()) std::iter_swap(terms.begin(), it);
  }
  row.seg[seg].insert(row.seg[seg].end(), terms.begin(), terms.end());
  if (!with_boundary) return;
  for (auto& kv : acc.cube) {
    if (g_drop_zeros && std::fabs(kv.second) <= 1e-12 * mxc) continue;
    HTerm t{std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
            std::get<4>(kv.first), std::get<5>(kv.first), std::get<6>(kv.first), kv.second};
    row.bseg[seg].push_back(t);
  }
}

}  // namespace

StencilSet build_stencils(int disc, double h, double nu_a, bool pspg_rhs) {
  const int ov = disc == HHG_P1P1_PSPG ? 1 : 2;
  const int G = ov == 1 ? 1 : 8;
  const int parr = 3 * G;
  const double nu_ah = nu_a * h;
  g_drop_zeros = nu_a == 0.0;
  ElemMats E[6];
  for (int s = 0; s < 6; ++s) E[s] = element_matrices(kuhn_tet(s), ov, h);
  const int nv = E[0].nv;
  auto K = [&](int s, int a, int b) { return E[s].K[a * nv + b]; };
  auto Mv = [&](int s, int a, int b) { return E[s].Mv[a * nv + b]; };
  auto Cq = [&](int s, int a, int b) { return E[s].Cq[a * 4 + b]; };
  auto Mq = [&](int s, int a, int b) { return E[s].Mq[a * 4 + b]; };
  auto MLq = [&](int s, int a, int b) {
    if (a != b) return 0.0;
    double r = 0;
    for (int l = 0; l < 4; ++l) r += E[s].Mq[a * 4 + l];
    return r;
  };

  StencilSet S;
  S.diagA.assign(G, 0.0);
  // ---------------- velocity rows
  for (int c = 0; c < 3; ++c)
    for (int g = 0; g < G; ++g) {
      const int out = c * G + g;
      BlockAcc aA, aBT, aM;
      accumulate_block(aA, ov, g, ov, c * G, +1, nu_ah, 1.0, K);
      accumulate_block(aBT, ov, g, 1, parr, 0, nu_ah, 1.0,
                       [&](int s, int a, int k) { return E[s].D[c][k * nv + a]; });
      accumulate_block(aM, ov, g, ov, c * G, 0, nu_ah, 1.0, Mv);
      HRow rA{out, g, false, {}, {}};
      flush_block(aA, rA, 1, true, c * G + g, false);
      HRow rBT{out, g, false, {}, {}};
      flush_block(aBT, rBT, 0, false, -1, false);
      HRow rF = rA;
      rF.seg[0] = rBT.seg[0];
      if (c == 0) S.diagA[g] = rA.seg[1].front().w;
      S.op[OP_A].rows.push_back(rA);
      S.op[OP_BT].rows.push_back(rBT);
      S.op[OP_FULL].rows.push_back(rF);
      HRow rM{out, g, true, {}, {}};
      flush_block(aM, rM, 0, false, -1, true);
      S.op[OP_MASS].rows.push_back(rM);
      HRow rMi{out, g, false, {}, {}};
      flush_block(aM, rMi, 0, false, -1, false);
      S.op[OP_MVINT].rows.push_back(rMi);
    }
  // ---------------- pressure rows
  {
    BlockAcc aB, aC, aMq, aL, aMLh, aML;
    for (int c = 0; c < 3; ++c) {
      accumulate_block(aB, 1, 0, ov, c * G, 0, nu_ah, 1.0, [&](int s, int k, int j) { return E[s].D[c][k * nv + j]; });
      if (ov == 1 && pspg_rhs)
        accumulate_block(aL, 1, 0, ov, c * G, -1, nu_ah, 1.0,
                         [&](int s, int k, int j) { return E[s].L[c][k * nv + j]; });
    }
    if (ov == 1) accumulate_block(aC, 1, 0, 1, parr, -1, nu_ah, 1.0, Cq);
    accumulate_block(aMq, 1, 0, 1, parr, 0, nu_ah, 1.0, Mq);
    accumulate_block(aMLh, 1, 0, 1, parr, -1, nu_ah, 1.0, MLq);
    accumulate_block(aML, 1, 0, 1, parr, 0, nu_ah, 1.0, MLq);
    HRow rB{parr, 0, true, {}, {}};
    flush_block(aB, rB, 0, false, -1, true);
    S.op[OP_B].rows.push_back(rB);
    HRow rBC = rB;                                   // B u - C p
    if (ov == 1) {
      HRow rC{parr, 0, true, {}, {}};
      flush_block(aC, rC, 2, false, -1, true);
      S.op[OP_C].rows.push_back(rC);
      rBC.seg[2] = rC.seg[2];
      rBC.bseg[2] = rC.bseg[2];
      for (auto& t : rBC.seg[2]) t.w = -t.w;
      for (auto& t : rBC.bseg[2]) t.w = -t.w;
    }
    S.op[OP_FULL].rows.push_back(rBC);
    S.op[OP_BC].rows.push_back(rBC);
    HRow rMq{parr, 0, true, {}, {}};
    flush_block(aMq, rMq, 0, false, -1, true);
    S.op[OP_MASS].rows.push_back(rMq);
    if (ov == 1 && pspg_rhs) {
      HRow rL{parr, 0, true, {}, {}};
      flush_block(aL, rL, 2, false, -1, true);
      S.op[OP_LOAD].rows.push_back(rL);
    }
    HRow rMLh{parr, 0, true, {}, {}};
    flush_block(aMLh, rMLh, 2, false, -1, true);
    S.op[OP_MLHAT].rows.push_back(rMLh);
    HRow rML{parr, 0, true, {}, {}};
    flush_block(aML, rML, 0, false, -1, true);
    S.op[OP_ML].rows.push_back(rML);
  }
  return S;
}

// ------------------------------------------------------------ transfers
HTransfer build_transfer(int order) {
  HTransfer X;
  X.order = order;
  const int G = order == 1 ? 1 : 8;
  const int span = order == 1 ? 2 : 4;        // fine positions per coarse cell
  X.nclass = span * span * span;
  X.prol.assign(X.nclass, {});
  X.restr.assign(G, {});
  std::map<std::tuple<int, int, int, int, int>, double> rmap;   // (gc, gf, ex, ey, ez) -> w
  for (int kz = 0; kz < span; ++kz)
    for (int ky = 0; ky < span; ++ky)
      for (int kx = 0; kx < span; ++kx) {
        const int kap[3] = {kx, ky, kz};
        const int cls = kx + span * (ky + span * kz);
        double t[3] = {double(kx) / span, double(ky) / span, double(kz) / span};
        // containing Kuhn tetrahedron: coordinates in descending order
        int p[3] = {0, 1, 2};
        std::stable_sort(p, p + 3, [&](int a, int b) { return t[a] > t[b]; });
        std::array<double, 4> lam = {1 - t[p[0]], t[p[0]] - t[p[1]], t[p[1]] - t[p[2]], t[p[2]]};
        int s = -1;
        for (int m = 0; m < 6; ++m)
          if (kPerm[m][0] == p[0] && kPerm[m][1] == p[1] && kPerm[m][2] == p[2]) s = m;
        Tet tet = kuhn_tet(s);
        std::vector<std::array<int, 3>> pos;
        local_positions(tet, order, pos);
        std::vector<double> phi;
        std::vector<std::array<double, 4>> dphi;
        basis(order, lam, phi, dphi);
        // fine group of this class
        int of[3], gf;
        if (order == 2) {
          for (int d = 0; d < 3; ++d) of[d] = kap[d] & 1;
          gf = group_of_parity(of[0], of[1], of[2]);
        } else {
          of[0] = of[1] = of[2] = 0;
          gf = 0;
        }
        for (size_t a = 0; a < pos.size(); ++a) {
          if (std::fabs(phi[a]) < 1e-14) continue;
          int oc[3] = {pos[a][0] & 1, pos[a][1] & 1, pos[a][2] & 1};
          int gc = group_of_parity(oc[0], oc[1], oc[2]);
          int dl[3] = {(pos[a][0] - oc[0]) / 2, (pos[a][1] - oc[1]) / 2, (pos[a][2] - oc[2]) / 2};
          X.prol[cls].push_back({gc, dl[0], dl[1], dl[2], phi[a]});
          int e[3];
          for (int d = 0; d < 3; ++d) e[d] = order == 2 ? -2 * dl[d] + (kap[d] - of[d]) / 2 : -2 * dl[d] + kap[d];
          rmap[{gc, gf, e[0], e[1], e[2]}] += phi[a];
        }
      }
  for (auto& kv : rmap) {
    int gc = std::get<0>(kv.first);
    X.restr[gc].push_back({std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first),
                           std::get<4>(kv.first), kv.second});
  }
  return X;
}

}  // namespace hhg
