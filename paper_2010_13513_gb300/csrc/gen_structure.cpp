// Build-time generator: prints the per-row term counts of the hot stencil
// operators (FULL, A, BT, BC) for P1-P1 / P2-P1 and constant / variable
// viscosity, as compile-time tables for the specialised kernels in fast.cu,
// and the pass/line plan of the streaming kernels in stream.cu.  The counts
// come from the same builder that produces the run-time weights, so the two
// always agree.
#include <algorithm>
#include <cstdio>
#include <map>
#include <set>
#include <vector>

#include "internal.h"

using namespace hhg;

// Plan of the streaming row kernels (stream.cu).  A pass stages a set of
// input arrays in shared memory plane by plane and evaluates every term that
// reads them.  Operators that read at most kPassArrays arrays take one pass;
// the others (P2-P1: FULL and (B, -C)) take one pass per velocity component
// (its G group arrays, plus the pressure array where a term of the pass reads
// it).  A row's terms may span passes (the pressure row of B u): its first
// pass writes it, later passes add to it.  Terms are listed by line
// (array slot, dj, dk) so that each line is loaded once per pass and plane.
constexpr int kPassArrays = 9;

void print_stream_plan(int disc, int varnu, int op, const HOperator& O) {
  struct Tm { int arr, di, dj, dk, row, seg, t; };
  std::vector<Tm> all;
  std::set<int> arrs;
  int t = 0;
  for (size_t r = 0; r < O.rows.size(); ++r)
    for (int sg = 0; sg < 3; ++sg)
      for (const HTerm& h : O.rows[r].seg[sg]) {
        all.push_back({h.in_arr, h.di, h.dj, h.dk, int(r), sg, t++});
        arrs.insert(h.in_arr);
      }
  const int G = disc == 2 ? 8 : 1, P = 3 * G;
  std::vector<std::vector<Tm>> passes;
  if (int(arrs.size()) <= kPassArrays) {
    passes.push_back(all);
  } else {
    passes.resize(3);
    for (const Tm& m : all) {
      const int out = O.rows[m.row].out_arr;
      int c = m.arr < P ? m.arr / G : (out < P ? out / G : 2);
      passes[c].push_back(m);
    }
  }
  // per row: first and last pass
  std::map<int, int> first, last;
  for (size_t q = 0; q < passes.size(); ++q)
    for (const Tm& m : passes[q]) {
      if (!first.count(m.row)) first[m.row] = int(q);
      last[m.row] = int(q);
    }
  std::vector<int> al;
  std::vector<std::vector<int>> pl;   // parts: {row, out, og, all, first, last}
  std::vector<std::vector<int>> ll;   // lines
  std::vector<std::vector<int>> el;   // terms
  std::vector<std::vector<int>> ps;
  int namax = 0, npmax = 0;
  for (size_t q = 0; q < passes.size(); ++q) {
    std::vector<Tm>& v = passes[q];
    std::set<int> pa;
    for (const Tm& m : v) pa.insert(m.arr);
    std::vector<int> slots(pa.begin(), pa.end());
    std::vector<int> rows;
    for (const Tm& m : v)
      if (std::find(rows.begin(), rows.end(), m.row) == rows.end()) rows.push_back(m.row);
    std::sort(rows.begin(), rows.end());
    auto slot_of = [&](int a) { return int(std::find(slots.begin(), slots.end(), a) - slots.begin()); };
    auto part_of = [&](int r) { return int(std::find(rows.begin(), rows.end(), r) - rows.begin()); };
    std::stable_sort(v.begin(), v.end(), [&](const Tm& a, const Tm& b) {
      const int sa = slot_of(a.arr), sb = slot_of(b.arr);
      if (sa != sb) return sa < sb;
      if (a.dk != b.dk) return a.dk < b.dk;
      if (a.dj != b.dj) return a.dj < b.dj;
      return a.di < b.di;
    });
    ps.push_back({int(al.size()), int(slots.size()), int(pl.size()), int(rows.size()), int(ll.size()), 0});
    for (int a : slots) al.push_back(a);
    for (int r : rows) {
      const HRow& R = O.rows[r];
      pl.push_back({r, R.out_arr, R.og, R.all_rows ? 1 : 0, first[r] == int(q) ? 1 : 0, last[r] == int(q) ? 1 : 0});
    }
    size_t i = 0;
    while (i < v.size()) {
      size_t j = i;
      int lmin = 1, lmax = -1;
      while (j < v.size() && v[j].arr == v[i].arr && v[j].dj == v[i].dj && v[j].dk == v[i].dk) {
        lmin = std::min(lmin, v[j].di);
        lmax = std::max(lmax, v[j].di);
        ++j;
      }
      ll.push_back({slot_of(v[i].arr), v[i].dj, v[i].dk, int(el.size()), int(j - i), lmin, lmax});
      for (size_t e = i; e < j; ++e) el.push_back({v[e].di, part_of(v[e].row), v[e].seg, v[e].t});
      i = j;
    }
    ps.back()[5] = int(ll.size()) - ps.back()[4];
    namax = std::max(namax, int(slots.size()));
    npmax = std::max(npmax, int(rows.size()));
  }
  auto list = [](const char* type, const char* name, const std::vector<std::vector<int>>& v) {
    std::printf("  static constexpr %s %s[%d] = {", type, name, int(v.size()));
    for (size_t i = 0; i < v.size(); ++i) {
      std::printf("%s{", i ? ", " : "");
      for (size_t k = 0; k < v[i].size(); ++k) std::printf("%s%d", k ? ", " : "", v[i][k]);
      std::printf("}");
    }
    std::printf("};\n");
  };
  // the C terms of the pressure row on the domain boundary: the distinct
  // lattice offsets of its per-cube terms (sorted by dk, dj, di); the library
  // sums the per-cube weights of every boundary class into this order
  std::vector<std::vector<int>> cbo;
  for (const HRow& R : O.rows)
    if (R.all_rows)
      for (const HTerm& h : R.bseg[2]) {
        std::vector<int> o = {h.di, h.dj, h.dk};
        if (std::find(cbo.begin(), cbo.end(), o) == cbo.end()) cbo.push_back(o);
      }
  std::sort(cbo.begin(), cbo.end(), [](const std::vector<int>& a, const std::vector<int>& b) {
    if (a[2] != b[2]) return a[2] < b[2];
    if (a[1] != b[1]) return a[1] < b[1];
    return a[0] < b[0];
  });
  std::printf("template <> struct SP<%d, %d, %d> {\n", disc, varnu, op);
  std::printf("  static constexpr int NCB = %d;\n", int(cbo.size()));
  if (!cbo.empty()) list("CubeO", "cbo", cbo);
  std::printf("  static constexpr int NP = %d, NAMAX = %d, NPMAX = %d, NL = %d, NE = %d;\n", int(passes.size()), namax,
              npmax, int(ll.size()), int(el.size()));
  list("PassT", "passes", ps);
  std::printf("  static constexpr int arrs[%d] = {", int(al.size()));
  for (size_t i = 0; i < al.size(); ++i) std::printf("%s%d", i ? ", " : "", al[i]);
  std::printf("};\n");
  list("PartT", "parts", pl);
  list("LineT", "lines", ll);
  list("TermE", "terms", el);
  // constant viscosity: the weights at h = 1 (weight index order); a term of
  // segment s scales as h^2 (s = 0: B, B^T), h (s = 1: A) or h^3 (s = 2: C)
  if (!varnu) {
    std::printf("  static constexpr double wref[%d] = {", int(all.size()));
    int n = 0;
    for (size_t r = 0; r < O.rows.size(); ++r)
      for (int sg = 0; sg < 3; ++sg)
        for (const HTerm& h : O.rows[r].seg[sg]) std::printf("%s%.17g", n++ ? ", " : "", h.w);
    std::printf("};\n");
  }
  std::printf("};\n");
}

int main() {
  std::printf("// generated by gen_structure.cpp -- do not edit\n#pragma once\nnamespace hhg {\nnamespace gen {\n");
  std::printf("struct RowS { int out, og, all, t0, n0, n1, n2; };\n");
  std::printf("template <int DISC, int VARNU, int OP> struct S;\n");
  // streaming-kernel plan (stream.cu): passes over staged input arrays
  std::printf("struct PassT { int a0, na, p0, np, l0, nl; };\n");
  std::printf("struct PartT { int row, out, og, all, first, last; };\n");
  std::printf("struct LineT { int slot, dj, dk, e0, ne, lmin, lmax; };\n");
  std::printf("struct TermE { int di, part, seg, t; };\n");
  std::printf("struct CubeO { int di, dj, dk; };\n");
  std::printf("template <int DISC, int VARNU, int OP> struct SP;\n");
  const int ops[4] = {OP_FULL, OP_A, OP_BT, OP_BC};
  for (int disc = 1; disc <= 2; ++disc)
    for (int varnu = 0; varnu <= 1; ++varnu) {
      StencilSet st = build_stencils(disc, 1.0, varnu ? 1.0 : 0.0, true);
      for (int op : ops) {
        const HOperator& O = st.op[op];
        int t = 0;
        std::printf("template <> struct S<%d, %d, %d> {\n  static constexpr int R = %d;\n", disc, varnu, op,
                    int(O.rows.size()));
        std::printf("  static constexpr RowS rows[%d] = {", int(O.rows.size()));
        for (size_t r = 0; r < O.rows.size(); ++r) {
          const HRow& R = O.rows[r];
          int n0 = int(R.seg[0].size()), n1 = int(R.seg[1].size()), n2 = int(R.seg[2].size());
          std::printf("%s{%d, %d, %d, %d, %d, %d, %d}", r ? ", " : "", R.out_arr, R.og, R.all_rows ? 1 : 0, t, n0, n1, n2);
          t += n0 + n1 + n2;
        }
        std::printf("};\n  static constexpr int N = %d;\n};\n", t);
        if (op == OP_A) continue;
        print_stream_plan(disc, varnu, op, O);
      }
    }
  std::printf("}  // namespace gen\n}  // namespace hhg\n");
  return 0;
}
