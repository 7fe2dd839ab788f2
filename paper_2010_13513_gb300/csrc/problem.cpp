// C ABI of the HHG Stokes library: meshes, problems, workspace binding and
// the solver drivers (Algorithm 1) issuing the CUDA kernels of kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "batch.h"
#include "dfres.h"
#include "fast.h"
#include "internal.h"
#include "kernels.h"
#include "nn.h"
#include "small.h"
#include "stream.h"

using namespace hhg;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define HHG_CUDA(call)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) return fail(HHG_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define HHG_CHECK_LAUNCH()                                                                      \
  do {                                                                                          \
    cudaError_t e_ = cudaGetLastError();                                                        \
    if (e_ != cudaSuccess) return fail(HHG_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e_)); \
  } while (0)

#define HHG_TRY(expr)          \
  do {                         \
    int rc_ = (expr);          \
    if (rc_ != HHG_OK) return rc_; \
  } while (0)

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

namespace hhg {
// records an error message for hhg_last_error (used by other translation units)
int set_error(int code, const std::string& msg) { return fail(code, msg); }
}  // namespace hhg

struct hhg_mesh {
  int mx, my, mz;
  double H;
};

namespace {

// serialised operator of one level
struct OpHost {
  std::vector<DRow> rows;
  std::vector<DTerm> terms;
  std::vector<double> w64;
  std::vector<DTermB> bterms;
  std::vector<double> bw64;
};

OpHost serialise(const HOperator& op, const Geo& g) {
  OpHost o;
  auto lin = [&](const HTerm& t) { return int(t.di + t.dj * g.sx + t.dk * g.sy); };
  for (const HRow& r : op.rows) {
    DRow d{};
    d.out_arr = r.out_arr; d.og = r.og; d.all_rows = r.all_rows ? 1 : 0;
    d.t0 = int(o.terms.size());
    int* ns[3] = {&d.n0, &d.n1, &d.n2};
    for (int s = 0; s < 3; ++s) {
      *ns[s] = int(r.seg[s].size());
      for (const HTerm& t : r.seg[s]) { o.terms.push_back({t.in_arr, lin(t)}); o.w64.push_back(t.w); }
    }
    d.b0 = int(o.bterms.size());
    int* ms[3] = {&d.m0, &d.m1, &d.m2};
    for (int s = 0; s < 3; ++s) {
      *ms[s] = int(r.bseg[s].size());
      for (const HTerm& t : r.bseg[s]) {
        o.bterms.push_back({t.in_arr, lin(t), t.cx, t.cy, t.cz, 0});
        o.bw64.push_back(t.w);
      }
    }
    o.rows.push_back(d);
  }
  return o;
}

struct Blob {                      // host staging of a device table region
  std::vector<char> bytes;
  template <class T>
  size_t put(const std::vector<T>& v) {
    size_t off = align256(bytes.size());
    bytes.resize(off + std::max<size_t>(v.size() * sizeof(T), 1));
    if (!v.empty()) std::memcpy(bytes.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
};

struct OpOffsets {
  size_t rows, terms, w64, w32, bterms, bw64, bw32;
  int nrows;
};

struct XferOffsets {
  size_t pstart, pterms, pw64, pw32, rstart, rterms, rw64, rw32;
  int order, nclass, ngroups, rmax;
};

struct Level {
  int l;
  Geo g;
  StencilSet st;
  OpOffsets opoff[OP_COUNT];
  OpDev op[OP_COUNT];
  std::vector<double> inv_diag;         // per group 1/diag(A)
  // parameter blocks of the specialised kernels (FastTab<T, N> images)
  std::vector<char> ftab64[OP_COUNT], ftab32[OP_COUNT];
  bool has_fast[OP_COUNT] = {};
  // parameter block of the double-float refinement residual (dfres.cu);
  // empty if the operator is not covered
  std::vector<char> dftab;
  // parameter blocks of the streaming kernels (FULL, B^T, (B, -C))
  std::vector<char> stab64[OP_COUNT], stab32[OP_COUNT];
  bool has_stream[OP_COUNT] = {};
  // parameter blocks (ResTabs images) of the shared-memory-resident
  // smoother, per CTA count (the offsets depend on the slab stride)
  std::map<int, std::vector<char>> rtab64, rtab32;
  int rctas[2] = {0, 0};                // CTAs of the resident smoother per precision (0: per-phase kernels)
  int rthreads[2] = {kResidentThreads, kResidentThreads};   // and threads per CTA
  Shape shape;                          // launch shapes of the specialised kernels
  // workspace offsets (bytes) of the level vectors
  size_t o_rhs, o_W, o_x64, o_tmp64, o_bw64, o_x32, o_b32, o_tmp32, o_invml, o_ml, o_esc;
  double *rhs = nullptr, *W = nullptr, *x64 = nullptr, *tmp64 = nullptr, *bw64 = nullptr;
  float *x32 = nullptr, *b32 = nullptr, *tmp32 = nullptr;
  double *inv_mlhat = nullptr, *ml = nullptr;
  double ml_sum = 0.0;
  int64_t nvec() const { return (3 * int64_t(g.G) + 1) * g.arr; }
  int64_t n_dofs() const;
  bool has_rhs = false;
};

}  // namespace

struct hhg_problem {
  hhg_mesh mesh;
  hhg_problem_desc desc;
  int G = 1, ov = 1;
  std::vector<Level> lv;               // levels lc .. L (+ L+1 if error_level)
  HTransfer tv, tp;
  XferOffsets xoff_v, xoff_p;
  XferDev xv{}, xp{};
  Blob tables;
  size_t o_tables = 0, o_Z = 0, o_idx = 0, o_part = 0, o_scal = 0, total = 0;
  int ncoarse = 0;
  char* ws = nullptr;
  double* Z = nullptr;
  int64_t* cidx = nullptr;
  double* partials = nullptr;
  double* scal = nullptr;               // device scalars
  int max_blocks = 1216;
  cudaStream_t stream = nullptr;
  bool bound = false;
  int64_t launches = 0;
  double wu_counted = 0.0;
  // CUDA graphs of whole FMG solves, keyed by the parameter tuple
  bool use_graphs = true;
  bool use_cluster = true;       // cluster-resident smoother on small levels
  int refine = HHG_REFINE_DF32;  // arithmetic of the mixed solve's refinement residual
  // learned coarse correction
  int nn_n = 0, nn_h = 0, nn_S = 0, nn_B = 0, nn_mode = 0;
  int64_t nn_P = 0;
  double nn_theta = 0.1;
  size_t o_nn = 0;
  float *nn_params = nullptr, *nn_grads = nullptr, *nn_m = nullptr, *nn_v = nullptr, *nn_Z = nullptr;
  float *nn_X = nullptr, *nn_T = nullptr, *nn_H1 = nullptr, *nn_H2 = nullptr, *nn_Y = nullptr, *nn_dY = nullptr;
  float *nn_dH1 = nullptr, *nn_dH2 = nullptr, *nn_xin = nullptr, *nn_h1 = nullptr, *nn_h2 = nullptr, *nn_y = nullptr;
  double *nn_mlp = nullptr, *nn_scal = nullptr, *nn_part = nullptr;
  float* nn_xyz = nullptr;       // coordinates and field of each coarse unknown (float4)
  unsigned long long* nn_counts = nullptr;
  int nn_step = 0;
  bool nn_recording = false;     // coarse solves append their defects to the samples
  double nn_tscale = 1.0;        // training targets are multiplied by this (unit RMS)

  struct Graph { cudaGraphExec_t exec; int64_t kernels; double wu; };
  // (parameter tuple, part: 0 whole solve, 1 stages below L, 2 stage L)
  std::map<std::tuple<int, int, int, int, int, int, double, int>, Graph> graphs;
  // second stream and events of hhg_fmg_solve_host (created on first use)
  cudaStream_t aux = nullptr, hp = nullptr;     // assembly; the FMG's stages at the highest priority
  cudaEvent_t ev_start = nullptr, ev_coarse = nullptr, ev_fine = nullptr, ev_done = nullptr;

  ~hhg_problem() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    for (cudaStream_t st : {aux, hp})
      if (st) cudaStreamDestroy(st);
    for (cudaEvent_t e : {ev_start, ev_coarse, ev_fine, ev_done})
      if (e) cudaEventDestroy(e);
  }

  Level& L(int l) { return lv[l - desc.coarse_level]; }
  int Lmax() const { return desc.L; }
};

int64_t Level::n_dofs() const {
  const int64_t np = int64_t(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
  const int64_t nv = g.G == 1 ? np : int64_t(2 * g.nx + 1) * (2 * g.ny + 1) * (2 * g.nz + 1);
  return 3 * nv + np;
}

// ===================================================================== misc
extern "C" int hhg_last_error(char* buf, size_t len) {
  if (!buf || len == 0) return HHG_EINVAL;
  std::snprintf(buf, len, "%s", g_err.c_str());
  return HHG_OK;
}

// =================================================================== meshes
extern "C" int hhg_mesh_create_box(int mx, int my, int mz, double H, hhg_mesh** out) {
  if (!out || mx < 1 || my < 1 || mz < 1 || !(H > 0)) return fail(HHG_EINVAL, "hhg_mesh_create_box: bad box");
  *out = new hhg_mesh{mx, my, mz, H};
  return HHG_OK;
}

extern "C" int hhg_mesh_create(const double* verts, int nv, const int* tets, int nt, hhg_mesh** out) {
  if (!verts || !tets || !out || nv < 4 || nt < 1) return fail(HHG_EINVAL, "hhg_mesh_create: bad arguments");
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int v = 0; v < nv; ++v)
    for (int d = 0; d < 3; ++d) { lo[d] = std::min(lo[d], verts[3 * v + d]); hi[d] = std::max(hi[d], verts[3 * v + d]); }
  for (int d = 0; d < 3; ++d)
    if (std::fabs(lo[d]) > 1e-12) return fail(HHG_EINVAL, "hhg_mesh_create: the box must start at the origin");
  // cube side: smallest positive coordinate step
  double H = 1e300;
  for (int t = 0; t < nt; ++t)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int d = 0; d < 3; ++d) {
          int va = tets[4 * t + a], vb = tets[4 * t + b];
          if (va < 0 || va >= nv || vb < 0 || vb >= nv) return fail(HHG_EINVAL, "hhg_mesh_create: vertex id out of range");
          double dd = std::fabs(verts[3 * va + d] - verts[3 * vb + d]);
          if (dd > 1e-12) H = std::min(H, dd);
        }
  int m[3];
  for (int d = 0; d < 3; ++d) {
    m[d] = int(std::lround(hi[d] / H));
    if (m[d] < 1 || std::fabs(m[d] * H - hi[d]) > 1e-9 * H) return fail(HHG_EINVAL, "hhg_mesh_create: not a box of cubes");
  }
  std::set<std::tuple<int, int, int, int, int, int>> seen;   // cube + path
  for (int t = 0; t < nt; ++t) {
    int c[4][3];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) {
        double q = verts[3 * tets[4 * t + a] + d] / H;
        c[a][d] = int(std::lround(q));
        if (std::fabs(q - c[a][d]) > 1e-9) return fail(HHG_EINVAL, "hhg_mesh_create: vertex off the cube lattice");
      }
    int order[4] = {0, 1, 2, 3};
    std::sort(order, order + 4, [&](int a, int b) { return c[a][0] + c[a][1] + c[a][2] < c[b][0] + c[b][1] + c[b][2]; });
    int dir[3];
    for (int s = 0; s < 3; ++s) {
      int dif[3], nz = 0, which = -1;
      for (int d = 0; d < 3; ++d) {
        dif[d] = c[order[s + 1]][d] - c[order[s]][d];
        if (dif[d] != 0) { ++nz; which = d; }
      }
      if (nz != 1 || dif[which] != 1) return fail(HHG_EINVAL, "hhg_mesh_create: tetrahedron is not a Kuhn simplex");
      dir[s] = which;
    }
    if (dir[0] == dir[1] || dir[1] == dir[2] || dir[0] == dir[2])
      return fail(HHG_EINVAL, "hhg_mesh_create: tetrahedron is not a Kuhn simplex");
    const int* o = c[order[0]];
    if (o[0] < 0 || o[1] < 0 || o[2] < 0 || o[0] >= m[0] || o[1] >= m[1] || o[2] >= m[2])
      return fail(HHG_EINVAL, "hhg_mesh_create: tetrahedron outside the box");
    seen.insert({o[0], o[1], o[2], dir[0], dir[1], dir[2]});
  }
  if (int64_t(seen.size()) != int64_t(6) * m[0] * m[1] * m[2] || nt != int(seen.size()))
    return fail(HHG_EINVAL, "hhg_mesh_create: the tetrahedra do not tile the box with 6 Kuhn simplices per cube");
  *out = new hhg_mesh{m[0], m[1], m[2], H};
  return HHG_OK;
}

extern "C" int hhg_mesh_destroy(hhg_mesh* mesh) {
  delete mesh;
  return HHG_OK;
}

// ================================================================= problems
extern "C" int hhg_problem_create(const hhg_mesh* mesh, const hhg_problem_desc* desc, hhg_problem** out) {
  if (!mesh || !desc || !out) return fail(HHG_EINVAL, "hhg_problem_create: null argument");
  if (desc->disc != HHG_P1P1_PSPG && desc->disc != HHG_P2P1_TH) return fail(HHG_EINVAL, "unknown discretisation");
  if (desc->L < 0 || desc->L > 10 || desc->coarse_level < 0 || desc->coarse_level > desc->L)
    return fail(HHG_EINVAL, "need 0 <= coarse_level <= L <= 10");
  if (desc->solve != HHG_SOLVE_FP64 && desc->solve != HHG_SOLVE_MIXED) return fail(HHG_EINVAL, "unknown solve mode");
  auto pb = std::make_unique<hhg_problem>();
  pb->mesh = *mesh;
  pb->desc = *desc;
  pb->ov = desc->disc == HHG_P1P1_PSPG ? 1 : 2;
  pb->G = pb->ov == 1 ? 1 : 8;
  const int top = desc->L + (desc->error_level ? 1 : 0);
  for (int l = desc->coarse_level; l <= top; ++l) {
    Level lv;
    lv.l = l;
    lv.g = make_geo(mesh->mx, mesh->my, mesh->mz, l, pb->G, mesh->H, desc->nu_a);
    if (int64_t(lv.g.nz + 1) * 25 > 65535 || lv.g.ny + 1 > 65535)
      return fail(HHG_EINVAL, "level too large for the launch geometry");
    lv.st = build_stencils(desc->disc, lv.g.h, desc->nu_a, desc->pspg_rhs != 0);
    for (int gg = 0; gg < pb->G; ++gg) lv.inv_diag.push_back(1.0 / lv.st.diagA[gg]);
    pb->lv.push_back(std::move(lv));
  }
  pb->tv = build_transfer(pb->ov);
  pb->tp = build_transfer(1);

  // ---- device table blob and specialised-kernel parameter blocks
  Blob& B = pb->tables;
  const int varnu = desc->nu_a != 0.0 ? 1 : 0;
  for (Level& lv : pb->lv) {
    for (int o = 0; o < OP_COUNT; ++o) {
      OpHost h = serialise(lv.st.op[o], lv.g);
      const int N = fast_terms(desc->disc, varnu, o);
      if (N >= 0) {
        if (N != int(h.terms.size())) return fail(HHG_EINVAL, "internal: specialised kernel structure mismatch");
        auto image = [&](auto zero, std::vector<char>& out) {
          using T = decltype(zero);
          const size_t bytes = (size_t(N) * (sizeof(T) + 4) + 7) / 8 * 8;
          out.assign(bytes, 0);
          T* w = reinterpret_cast<T*>(out.data());
          int* off = reinterpret_cast<int*>(out.data() + size_t(N) * sizeof(T));
          for (int t = 0; t < N; ++t) {
            const int64_t lin = int64_t(h.terms[t].arr) * lv.g.arr + h.terms[t].off;
            if (lin > INT32_MAX || lin < INT32_MIN) return false;
            w[t] = T(h.w64[t]);
            off[t] = int(lin);
          }
          return true;
        };
        if (!image(0.0, lv.ftab64[o]) || !image(0.0f, lv.ftab32[o])) return fail(HHG_EINVAL, "level too large for 32-bit offsets");
        lv.has_fast[o] = true;
        if (o == OP_FULL) df_table(desc->disc, varnu, lv.ftab64[o], lv.dftab);
      }
      if (N >= 0 && (o == OP_FULL || o == OP_BT || o == OP_BC)) {
        // streaming kernels: the weights, and the boundary C stencil of the
        // pressure row summed per boundary class (27 classes: each of i, j, k
        // on the low face, inside, or on the high face; a per-cube term
        // counts where its cube lies inside the box)
        std::vector<int> offs;
        stream_c_offsets(desc->disc, varnu, o, offs);
        const int ncb = int(offs.size()) / 3;
        std::vector<double> wc(size_t(27) * ncb, 0.0);
        for (const HRow& R : lv.st.op[o].rows)
          if (R.all_rows)
            for (const HTerm& t : R.bseg[2]) {
              int slot = -1;
              for (int q = 0; q < ncb; ++q)
                if (offs[3 * q] == t.di && offs[3 * q + 1] == t.dj && offs[3 * q + 2] == t.dk) slot = q;
              if (slot < 0) return fail(HHG_EINVAL, "internal: boundary stencil offset missing from the plan");
              const int cc[3] = {t.cx, t.cy, t.cz};
              for (int cls = 0; cls < 27; ++cls) {
                const int c3[3] = {cls % 3, (cls / 3) % 3, cls / 9};
                bool in = true;
                for (int d = 0; d < 3; ++d) in = in && !(c3[d] == 0 && cc[d] < 0) && !(c3[d] == 2 && cc[d] >= 0);
                if (in) wc[size_t(cls) * ncb + slot] += t.w;
              }
            }
        lv.has_stream[o] = stream_image<double>(desc->disc, varnu, o, h.w64, wc, lv.stab64[o]) &&
                           stream_image<float>(desc->disc, varnu, o, h.w64, wc, lv.stab32[o]);
      }
      std::vector<float> w32(h.w64.begin(), h.w64.end()), bw32(h.bw64.begin(), h.bw64.end());
      OpOffsets& of = lv.opoff[o];
      of.nrows = int(h.rows.size());
      of.rows = B.put(h.rows); of.terms = B.put(h.terms); of.w64 = B.put(h.w64); of.w32 = B.put(w32);
      of.bterms = B.put(h.bterms); of.bw64 = B.put(h.bw64); of.bw32 = B.put(bw32);
    }
  }
  auto put_x = [&](const HTransfer& X, XferOffsets& xo) {
    std::vector<int> ps(1, 0), rs(1, 0);
    std::vector<DXTerm> pt, rt;
    std::vector<double> pw, rw;
    for (auto& c : X.prol) {
      for (auto& t : c) { pt.push_back({t.arr, t.di, t.dj, t.dk}); pw.push_back(t.w); }
      ps.push_back(int(pt.size()));
    }
    for (auto& c : X.restr) {
      for (auto& t : c) { rt.push_back({t.arr, t.di, t.dj, t.dk}); rw.push_back(t.w); }
      rs.push_back(int(rt.size()));
    }
    std::vector<float> pw32(pw.begin(), pw.end()), rw32(rw.begin(), rw.end());
    xo.order = X.order; xo.nclass = X.nclass; xo.ngroups = int(X.restr.size());
    xo.rmax = 0;
    for (auto& c : X.restr) xo.rmax = std::max(xo.rmax, int(c.size()));
    xo.pstart = B.put(ps); xo.pterms = B.put(pt); xo.pw64 = B.put(pw); xo.pw32 = B.put(pw32);
    xo.rstart = B.put(rs); xo.rterms = B.put(rt); xo.rw64 = B.put(rw); xo.rw32 = B.put(rw32);
  };
  put_x(pb->tv, pb->xoff_v);
  put_x(pb->tp, pb->xoff_p);

  // ---- workspace layout
  size_t off = 0;
  pb->o_tables = off;
  off = align256(off + B.bytes.size());
  const bool mixed = desc->solve == HHG_SOLVE_MIXED;
  for (Level& lv : pb->lv) {
    const size_t v64 = align256(size_t(lv.nvec()) * 8), v32 = align256(size_t(lv.nvec()) * 4);
    const size_t a64 = align256(size_t(lv.g.arr) * 8);
    lv.o_rhs = off; off += v64;
    lv.o_W = off; off += v64;
    lv.o_x64 = off; off += v64;
    lv.o_tmp64 = off; off += v64;
    lv.o_bw64 = off; off += v64;
    if (mixed) {
      lv.o_x32 = off; off += v32;
      lv.o_b32 = off; off += v32;
      lv.o_tmp32 = off; off += v32;
    }
    lv.o_invml = off; off += a64;
    lv.o_ml = off; off += a64;
    lv.o_esc = off; off += align256(size_t(2 * (lv.g.nz + 1)) * 8);
  }
  // coarse system: interior velocity DoFs of the coarse level + all pressure nodes
  {
    const Geo& g = pb->lv[0].g;
    int n = 0;
    for (int gg = 0; gg < pb->G; ++gg) {
      const int* o = kGroupOff[gg];
      for (int k = 0; k <= g.nz - o[2]; ++k)
        for (int j = 0; j <= g.ny - o[1]; ++j)
          for (int i = 0; i <= g.nx - o[0]; ++i) {
            int P[3] = {2 * i + o[0], 2 * j + o[1], 2 * k + o[2]};
            bool bnd = P[0] == 0 || P[1] == 0 || P[2] == 0 || P[0] == 2 * g.nx || P[1] == 2 * g.ny || P[2] == 2 * g.nz;
            if (!bnd) ++n;
          }
    }
    n = 3 * n + (g.nx + 1) * (g.ny + 1) * (g.nz + 1);
    if (n > 6000) return fail(HHG_EINVAL, "coarse level too large for the dense coarse solve");
    pb->ncoarse = n;
  }
  pb->o_Z = off; off += align256(size_t(pb->ncoarse) * pb->ncoarse * 8);
  pb->o_idx = off; off += align256(size_t(pb->ncoarse) * 8);
  pb->o_part = off; off += align256(size_t(pb->max_blocks) * 8);
  pb->o_scal = off; off += align256(64 * 8);
  if (desc->nn_hidden > 0) {
    if (desc->nn_samples < 2 || desc->nn_batch < 1) return fail(HHG_EINVAL, "nn_samples >= 2 and nn_batch >= 1 needed");
    const int n = pb->ncoarse, h = desc->nn_hidden;
    pb->nn_n = n; pb->nn_h = h; pb->nn_S = desc->nn_samples; pb->nn_B = desc->nn_batch;
    pb->nn_P = int64_t(h) * n + h + int64_t(h) * h + h + int64_t(n) * h + n;
    const int64_t B = std::max(desc->nn_batch, 1);
    const int64_t floats = 4 * pb->nn_P + int64_t(n) * n + 2 * int64_t(pb->nn_S) * n + 4 * B * h + 2 * B * n +
                           6 * int64_t(n) + 2 * int64_t(h) + 4;
    pb->o_nn = off;
    off += align256(size_t(floats) * 4) + align256(size_t(n) * 8) + align256(64 * 8) + align256(1024 * 8) + 256;
  }
  pb->total = off;
  *out = pb.release();
  return HHG_OK;
}

extern "C" int hhg_problem_workspace_bytes(const hhg_problem* pb, size_t* bytes) {
  if (!pb || !bytes) return fail(HHG_EINVAL, "null argument");
  *bytes = pb->total;
  return HHG_OK;
}

extern "C" int hhg_problem_destroy(hhg_problem* pb) {
  delete pb;
  return HHG_OK;
}

extern "C" int hhg_layout(const hhg_problem* pb, int level, hhg_layout_info* info) {
  if (!pb || !info) return fail(HHG_EINVAL, "null argument");
  const int top = pb->desc.L + (pb->desc.error_level ? 1 : 0);
  if (level < pb->desc.coarse_level || level > top) return fail(HHG_EINVAL, "level out of range");
  const Level& lv = pb->lv[level - pb->desc.coarse_level];
  const Geo& g = lv.g;
  info->level = level;
  info->nx = g.nx; info->ny = g.ny; info->nz = g.nz;
  info->groups = g.G;
  info->sx = g.sx; info->sy = g.sy;
  info->array_elems = g.arr;
  info->vector_elems = lv.nvec();
  info->n_pressure_nodes = int64_t(g.nx + 1) * (g.ny + 1) * (g.nz + 1);
  info->n_velocity_nodes = g.G == 1 ? info->n_pressure_nodes : int64_t(2 * g.nx + 1) * (2 * g.ny + 1) * (2 * g.nz + 1);
  info->n_dofs = 3 * info->n_velocity_nodes + info->n_pressure_nodes;
  info->h = g.h;
  return HHG_OK;
}

// ------------------------------------------------------- layout conversion
namespace {

// canonical index -> (array, site) for velocity nodes of level geometry g
template <class F>
void for_each_velocity_node(const Geo& g, F f) {
  if (g.G == 1) {
    int64_t c = 0;
    for (int k = 0; k <= g.nz; ++k)
      for (int j = 0; j <= g.ny; ++j)
        for (int i = 0; i <= g.nx; ++i, ++c)
          f(c, 0, int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy, i == 0 || j == 0 || k == 0 || i == g.nx || j == g.ny || k == g.nz);
  } else {
    int64_t c = 0;
    for (int K = 0; K <= 2 * g.nz; ++K)
      for (int J = 0; J <= 2 * g.ny; ++J)
        for (int I = 0; I <= 2 * g.nx; ++I, ++c) {
          int gg = group_of_parity(I & 1, J & 1, K & 1);
          f(c, gg, int64_t((I >> 1) + 1) + int64_t((J >> 1) + 1) * g.sx + int64_t((K >> 1) + 1) * g.sy,
            I == 0 || J == 0 || K == 0 || I == 2 * g.nx || J == 2 * g.ny || K == 2 * g.nz);
        }
  }
}

template <class F>
void for_each_pressure_node(const Geo& g, F f) {
  int64_t c = 0;
  for (int k = 0; k <= g.nz; ++k)
    for (int j = 0; j <= g.ny; ++j)
      for (int i = 0; i <= g.nx; ++i, ++c) f(c, int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy);
}

int check_prec(const hhg_problem* pb, int prec) {
  if (prec == HHG_FP64) return HHG_OK;
  if (prec == HHG_FP32 && pb->desc.solve == HHG_SOLVE_MIXED) return HHG_OK;
  return fail(HHG_EINVAL, "FP32 operations need a problem created with HHG_SOLVE_MIXED");
}

int check_level(const hhg_problem* pb, int level, bool allow_error_level = false) {
  if (!pb) return fail(HHG_EINVAL, "null problem");
  if (!pb->bound) return fail(HHG_ESTATE, "problem has no workspace bound (call hhg_problem_bind)");
  const int top = pb->desc.L + ((allow_error_level && pb->desc.error_level) ? 1 : 0);
  if (level < pb->desc.coarse_level || level > top) return fail(HHG_EINVAL, "level out of range");
  return HHG_OK;
}

}  // namespace

namespace {
int64_t velocity_nodes(const Geo& g) {
  return g.G == 1 ? int64_t(g.nx + 1) * (g.ny + 1) * (g.nz + 1)
                  : int64_t(2 * g.nx + 1) * (2 * g.ny + 1) * (2 * g.nz + 1);
}
int64_t pressure_nodes(const Geo& g) { return int64_t(g.nx + 1) * (g.ny + 1) * (g.nz + 1); }
}  // namespace

// Canonical host data cross the bus as they are (one copy each way, fast from
// pinned host memory) and are scattered to / gathered from the padded layout
// on the device, staged in the level's scratch vector bw64.
extern "C" int hhg_vector_from_host(hhg_problem* pb, int level, int prec, const double* host, void* dev) {
  HHG_TRY(check_level(pb, level, true));
  HHG_TRY(check_prec(pb, prec));
  if (!host || !dev) return fail(HHG_EINVAL, "null vector");
  Level& lv = pb->L(level);
  const int64_t nvn = velocity_nodes(lv.g), npn = pressure_nodes(lv.g);
  HHG_CUDA(cudaMemcpyAsync(lv.bw64, host, size_t(3 * nvn + npn) * 8, cudaMemcpyHostToDevice, pb->stream));
  if (prec == HHG_FP64) {
    HHG_CUDA(cudaMemsetAsync(dev, 0, size_t(lv.nvec()) * 8, pb->stream));
    launch_canon_scatter<double>(lv.g, lv.bw64, static_cast<double*>(dev), nvn, npn, true, false, pb->stream);
  } else {
    HHG_CUDA(cudaMemsetAsync(dev, 0, size_t(lv.nvec()) * 4, pb->stream));
    launch_canon_scatter<float>(lv.g, lv.bw64, static_cast<float*>(dev), nvn, npn, true, false, pb->stream);
  }
  HHG_CHECK_LAUNCH();
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  return HHG_OK;
}

extern "C" int hhg_vector_to_host(hhg_problem* pb, int level, int prec, const void* dev, double* host) {
  HHG_TRY(check_level(pb, level, true));
  HHG_TRY(check_prec(pb, prec));
  if (!host || !dev) return fail(HHG_EINVAL, "null vector");
  Level& lv = pb->L(level);
  const int64_t nvn = velocity_nodes(lv.g), npn = pressure_nodes(lv.g);
  if (prec == HHG_FP64) launch_canon_gather<double>(lv.g, static_cast<const double*>(dev), lv.bw64, nvn, npn, pb->stream);
  else launch_canon_gather<float>(lv.g, static_cast<const float*>(dev), lv.bw64, nvn, npn, pb->stream);
  HHG_CHECK_LAUNCH();
  HHG_CUDA(cudaMemcpyAsync(host, lv.bw64, size_t(3 * nvn + npn) * 8, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  return HHG_OK;
}

// ============================================================ solver steps
namespace {

template <class T> T* vx(Level& lv);
template <> double* vx<double>(Level& lv) { return lv.x64; }
template <> float* vx<float>(Level& lv) { return lv.x32; }
template <class T> T* vb(Level& lv);
template <> double* vb<double>(Level& lv) { return lv.bw64; }
template <> float* vb<float>(Level& lv) { return lv.b32; }
template <class T> T* vt(Level& lv);
template <> double* vt<double>(Level& lv) { return lv.tmp64; }
template <> float* vt<float>(Level& lv) { return lv.tmp32; }

int64_t p_offset(const Level& lv) { return 3 * int64_t(lv.g.G) * lv.g.arr; }

// relative cost of one block application (paper's normalisation, Sec. 4.2)
struct Costs { double A, B, C; };
Costs block_costs(int ov) {
  if (ov == 2) return {46.0 / 72, 13.0 / 72, 0.0};
  return {0.3, 0.3, 0.1};
}

template <class T> const void* ftab(Level& lv, int op);
template <> const void* ftab<double>(Level& lv, int op) { return lv.ftab64[op].data(); }
template <> const void* ftab<float>(Level& lv, int op) { return lv.ftab32[op].data(); }

template <class T> const void* stab(Level& lv, int op);
template <> const void* stab<double>(Level& lv, int op) { return lv.stab64[op].data(); }
template <> const void* stab<float>(Level& lv, int op) { return lv.stab32[op].data(); }

// the streaming kernels of op if the level's shape selects them (true if launched)
template <class T>
bool stream_op(hhg_problem* pb, Level& lv, const Shape& sh, int op, int mode, const T* x, const T* b, T* y) {
  const int si = op == OP_FULL ? 0 : op == OP_BT ? 1 : op == OP_BC ? 2 : -1;
  if (si < 0 || mode == MODE_ADD || !lv.has_stream[op]) return false;
  const int nt = sizeof(T) == 8 ? sh.st64_threads[si] : sh.st_threads[si];
  const int ns = sizeof(T) == 8 ? 4 : sh.st_sites[si];
  if (!nt) return false;
  const int disc = pb->desc.disc, varnu = pb->desc.nu_a != 0.0 ? 1 : 0;
  return stream_rows<T>(disc, varnu, op, mode, lv.g, stab<T>(lv, op), x, b, y, nt, ns, pb->stream);
}

template <class T>
int apply_op(hhg_problem* pb, Level& lv, int op, int mode, const T* x, const T* b, T* y, double alpha = 1.0) {
  if (stream_op<T>(pb, lv, lv.shape, op, mode, x, b, y)) {
    HHG_CHECK_LAUNCH();
    return HHG_OK;
  }
  if (lv.has_fast[op] && op != OP_A)
    fast_rows<T>(pb->desc.disc, pb->desc.nu_a != 0.0 ? 1 : 0, op, lv.g, lv.op[op], ftab<T>(lv, op), mode, x, b, y,
                 alpha, lv.shape, pb->stream);
  else
    launch_apply<T>(lv.g, lv.op[op], mode, x, b, y, alpha, pb->stream);
  HHG_CHECK_LAUNCH();
  return HHG_OK;
}

double level_weight(hhg_problem* pb, const Level& lv) {
  return double(lv.n_dofs()) / double(pb->L(pb->desc.L).n_dofs());
}

template <class T> constexpr int prec_index() { return sizeof(T) == 8 ? HHG_FP64 : HHG_FP32; }
template <class T> const ResTabs<T>& rtab(Level& lv, int C);
template <> const ResTabs<double>& rtab<double>(Level& lv, int C) {
  return *reinterpret_cast<const ResTabs<double>*>(lv.rtab64.at(C).data());
}
template <> const ResTabs<float>& rtab<float>(Level& lv, int C) {
  return *reinterpret_cast<const ResTabs<float>*>(lv.rtab32.at(C).data());
}

// true if a linear offset di + dj sx + dk sy reaches only adjacent sites
bool adjacent(const Geo& g, int64_t off) {
  const int64_t dk = std::llround(double(off) / double(g.sy));
  const int64_t dj = std::llround(double(off - dk * g.sy) / double(g.sx));
  const int64_t di = off - dk * g.sy - dj * g.sx;
  return dk >= -1 && dk <= 1 && dj >= -1 && dj <= 1 && di >= -1 && di <= 1;
}

// the resident smoother's parameter block for slab stride arr_l: rows and
// terms of A (component 0 of each group), B^T and (B, -C) from the level's
// stencil tables, offsets rewritten to the slab stride
template <class T>
int build_res_tabs(hhg_problem* pb, Level& lv, int64_t arr_l, std::vector<char>& out) {
  out.assign(sizeof(ResTabs<T>), 0);
  ResTabs<T>& rt = *reinterpret_cast<ResTabs<T>*>(out.data());
  const int G = lv.g.G;
  rt.G = G;
  rt.nbt = 3 * G;
  rt.varnu = pb->desc.nu_a != 0.0 ? 1 : 0;
  const char* blob = pb->tables.bytes.data();
  int nw = 0;
  auto add = [&](int op, int r, ResRow& dst) {
    const OpOffsets& of = lv.opoff[op];
    if (r >= of.nrows) return false;
    const DRow& d = reinterpret_cast<const DRow*>(blob + of.rows)[r];
    const DTerm* terms = reinterpret_cast<const DTerm*>(blob + of.terms);
    const double* w = reinterpret_cast<const double*>(blob + of.w64);
    const int n = d.n0 + d.n1 + d.n2;
    if (nw + n > kResMaxTerms) return false;
    dst = ResRow{d.out_arr, d.og, d.all_rows, nw, d.n0, d.n1, d.n2, d.b0 + d.m0 + d.m1, d.m2};
    for (int t = d.t0; t < d.t0 + n; ++t) {
      if (terms[t].arr < 0 || terms[t].arr > 3 * G || !adjacent(lv.g, terms[t].off)) return false;
      rt.w[nw] = T(w[t]);
      rt.off[nw] = int(terms[t].arr * arr_l + terms[t].off);
      ++nw;
    }
    return true;
  };
  bool ok = G <= 8 && 3 * G <= kResMaxRows;
  for (int gg = 0; ok && gg < G; ++gg) {
    ok = add(OP_A, gg, rt.A[gg]);
    ok = ok && rt.A[gg].n0 == 0 && rt.A[gg].n2 == 0 && rt.A[gg].n1 > 0;   // diagonal first, all in segment 1
  }
  for (int r = 0; ok && r < 3 * G; ++r) ok = add(OP_BT, r, rt.BT[r]);
  ok = ok && add(OP_BC, 0, rt.BC);
  if (!ok) return fail(HHG_EINVAL, "internal: stencil tables do not fit the resident smoother");
  rt.nw = nw;
  return HHG_OK;
}

// selects `ctas` CTAs (0: per-phase kernels) for the resident smoother of a
// level in precision `prec`; HHG_EINVAL if the level does not fit
int set_resident(hhg_problem* pb, Level& lv, int prec, int ctas, int threads = kResidentThreads) {
  if (ctas < 0 || ctas > kResidentMaxCtas) return fail(HHG_EINVAL, "ctas must be in 0..16");
  if (threads < 128 || threads > kResidentThreads || threads % 32)
    return fail(HHG_EINVAL, "threads must be a multiple of 32 in 128..1024");
  if (ctas > 0) {
    if (!resident_feasible(prec, lv.g, ctas))
      return fail(HHG_EINVAL, "level does not fit the shared memory of that many CTAs");
    // the per-cube boundary terms of (B, -C) must stay within the adjacent
    // sites, as the slab holds one halo plane on each side
    const OpOffsets& of = lv.opoff[OP_BC];
    const DRow* rows = reinterpret_cast<const DRow*>(pb->tables.bytes.data() + of.rows);
    const DTermB* bt = reinterpret_cast<const DTermB*>(pb->tables.bytes.data() + of.bterms);
    for (int r = 0; r < of.nrows; ++r)
      for (int t = rows[r].b0; t < rows[r].b0 + rows[r].m0 + rows[r].m1 + rows[r].m2; ++t) {
        const int64_t dk = std::llround(double(bt[t].off) / double(lv.g.sy));
        const int64_t dj = std::llround(double(bt[t].off - dk * lv.g.sy) / double(lv.g.sx));
        const int64_t di = bt[t].off - dk * lv.g.sy - dj * lv.g.sx;
        if (bt[t].arr < 0 || bt[t].arr > 3 * lv.g.G || dk < -1 || dk > 1 || dj < -1 || dj > 1 || di < -1 || di > 1)
          return fail(HHG_EINVAL, "internal: boundary stencil offsets beyond adjacent sites");
      }
    auto& cache = prec == HHG_FP64 ? lv.rtab64 : lv.rtab32;
    if (!cache.count(ctas)) {
      std::vector<char> img;
      if (prec == HHG_FP64) HHG_TRY(build_res_tabs<double>(pb, lv, resident_arr(lv.g, ctas), img));
      else HHG_TRY(build_res_tabs<float>(pb, lv, resident_arr(lv.g, ctas), img));
      cache[ctas] = std::move(img);
    }
  }
  lv.rctas[prec] = ctas;
  lv.rthreads[prec] = threads;
  return HHG_OK;
}

// default CTA count: the fewest CTAs (at most 8) that hold the level with at
// most 8192 lattice sites each, else none (per-phase kernels)
int default_resident(hhg_problem* pb, Level& lv, int prec) {
  const int64_t plane = int64_t(lv.g.nx + 1) * (lv.g.ny + 1), nzp = lv.g.nz + 1;
  for (int C : {1, 2, 4, 8})
    if (plane * ((nzp + C - 1) / C) <= 8192 && resident_feasible(prec, lv.g, C))
      return set_resident(pb, lv, prec, C);
  return set_resident(pb, lv, prec, 0);
}

template <class T>
int uzawa(hhg_problem* pb, Level& lv, const hhg_params& prm, int sweeps, T* x, const T* b, T* tmp) {
  const int G = lv.g.G;
  if (sweeps <= 0) return HHG_OK;
  const int C = lv.rctas[prec_index<T>()];
  if (C > 0 && pb->use_cluster) {
    // all phases of all sweeps in one cluster launch, the level in shared memory
    SmallArgs a{};
    a.iterations = sweeps;
    a.xi = prm.xi;
    a.ahat = prm.ahat;
    a.inv_omega_inv = 1.0 / prm.omega_inv;
    for (int gg = 0; gg < G; ++gg) a.inv_diag[gg] = lv.inv_diag[gg];
    if (uzawa_resident<T>(lv.g, C, lv.rthreads[prec_index<T>()], x, b, lv.inv_mlhat, a, lv.op[OP_BC], rtab<T>(lv, C),
                          pb->stream) != 0)
      return fail(HHG_ECUDA, std::string("resident smoother launch: ") + cudaGetErrorString(cudaGetLastError()));
    const Costs cs = block_costs(pb->ov);
    pb->wu_counted += sweeps * level_weight(pb, lv) * (prm.xi * (prm.ahat == HHG_AHAT_S ? 2 : 1) * cs.A + 2 * cs.B + cs.C);
    return HHG_OK;
  }
  std::vector<std::pair<int, int>> phases;
  for (int c = 0; c < 4; ++c) phases.push_back({0, c});
  for (int gg = 1; gg < G; ++gg) phases.push_back({gg, -1});
  const Costs cs = block_costs(pb->ov);
  for (int it = 0; it < sweeps; ++it) {
    // velocity step (Eq. uzawa-velocity): f' = f - B^T p_k, xi GS sweeps on A u = f'
    HHG_TRY(apply_op<T>(pb, lv, OP_BT, MODE_RES, x, b, tmp));
    const int disc = pb->desc.disc, varnu = pb->desc.nu_a != 0.0 ? 1 : 0;
    const void* tabA = ftab<T>(lv, OP_A);
    // A is block diagonal over the velocity components: either every phase
    // on all three components, or all sweeps of one component after another
    // (the same iterates)
    const bool cm = lv.shape.gs_comp_major != 0;
    for (int c = cm ? 0 : -1; c < (cm ? 3 : 0); ++c)
      for (int s = 0; s < prm.xi; ++s) {
        for (auto& ph : phases)
          fast_gs<T>(disc, varnu, lv.g, tabA, ph.first, ph.second, lv.inv_diag[ph.first], x, tmp, lv.shape, pb->stream,
                     c);
        if (prm.ahat == HHG_AHAT_S)
          for (auto it2 = phases.rbegin(); it2 != phases.rend(); ++it2)
            fast_gs<T>(disc, varnu, lv.g, tabA, it2->first, it2->second, lv.inv_diag[it2->first], x, tmp, lv.shape,
                       pb->stream, c);
      }
    HHG_CHECK_LAUNCH();
    // pressure step (Eq. uzawa-pressure): p -= S_hat^{-1} (g - B u_{k+1} + C p_k)
    HHG_TRY(apply_op<T>(pb, lv, OP_BC, MODE_RES, x, b, tmp));
    const int64_t po = p_offset(lv);
    launch_pupdate<T>(lv.g, x + po, tmp + po, lv.inv_mlhat, 1.0 / prm.omega_inv, pb->stream);
    HHG_CHECK_LAUNCH();
    pb->wu_counted += level_weight(pb, lv) * (prm.xi * (prm.ahat == HHG_AHAT_S ? 2 : 1) * cs.A + 2 * cs.B + cs.C);
  }
  return HHG_OK;
}

template <class T>
int restrict_to(hhg_problem* pb, int l, const T* rf, T* rc) {
  Level& f = pb->L(l);
  Level& c = pb->L(l - 1);
  launch_restrict<T>(f.g, c.g, pb->xv, 0, 0, 3, pb->G, true, rf, rc, pb->stream);
  launch_restrict<T>(f.g, c.g, pb->xp, 3 * pb->G, 3 * pb->G, 1, 1, false, rf, rc, pb->stream);
  HHG_CHECK_LAUNCH();
  return HHG_OK;
}

template <class T>
int prolong_add(hhg_problem* pb, int l, const T* xc, T* xf, bool velocity_interior_only = true) {
  Level& f = pb->L(l);
  Level& c = pb->L(l - 1);
  launch_prolong<T>(f.g, c.g, pb->xv, 0, 0, 3, pb->G, velocity_interior_only, xc, xf, pb->stream);
  launch_prolong<T>(f.g, c.g, pb->xp, 3 * pb->G, 3 * pb->G, 1, 1, false, xc, xf, pb->stream);
  HHG_CHECK_LAUNCH();
  return HHG_OK;
}

template <class T> int coarse_nn(hhg_problem* pb, const T* b, T* x);

template <class T>
int coarse_solve(hhg_problem* pb, const T* b, T* x) {
  Level& lv = pb->lv[0];
  HHG_CUDA(launch_zero(x, size_t(lv.nvec()) * sizeof(T), pb->stream));
  if (pb->nn_recording) {
    nn_gather<T>(b, pb->cidx, pb->nn_n, pb->nn_xin, pb->nn_scal, pb->stream);
    nn_record(pb->nn_xin, pb->nn_X, pb->nn_n, pb->nn_S, pb->nn_counts + 2, pb->stream);
  }
  if (pb->nn_mode == 3) return HHG_OK;            // comparison mode: no coarse correction
  if (pb->nn_mode != 0) return coarse_nn<T>(pb, b, x);
  launch_coarse<T>(pb->Z, pb->ncoarse, pb->cidx, b, x, pb->stream);
  HHG_CHECK_LAUNCH();
  return HHG_OK;
}

template <class T>
int residual(hhg_problem* pb, Level& lv, const T* x, const T* b, T* r) {
  HHG_TRY(apply_op<T>(pb, lv, OP_FULL, MODE_RES, x, b, r));
  pb->wu_counted += level_weight(pb, lv);
  return HHG_OK;
}

// the defect of the mixed solve's refinement step, r32 = fl32(b - calA x):
// the double-float kernels where they cover the operator (x32 and tmp64
// serve as scratch for the two FP32 parts of x), else the FP64 residual in
// tmp64 rounded to FP32
int refinement_residual(hhg_problem* pb, Level& lv, const double* x, const double* b, float* r32) {
  if (pb->refine == HHG_REFINE_DF32 && !lv.dftab.empty()) {
    df_residual(pb->desc.disc, pb->desc.nu_a != 0.0 ? 1 : 0, lv.g, lv.op[OP_FULL], lv.dftab, x, b, lv.x32,
                reinterpret_cast<float*>(lv.tmp64), r32, pb->stream);
    HHG_CHECK_LAUNCH();
    pb->wu_counted += level_weight(pb, lv);
    return HHG_OK;
  }
  HHG_TRY(residual<double>(pb, lv, x, b, lv.tmp64));
  launch_cast_d2f(lv.tmp64, r32, lv.nvec(), pb->stream);
  HHG_CHECK_LAUNCH();
  return HHG_OK;
}

// VAR-V-CYCLE(l_fine, l, ...) of Algorithm 1
template <class T>
int vcycle(hhg_problem* pb, int lf, int l, const hhg_params& prm, T* x, const T* b) {
  if (l == pb->desc.coarse_level) return coarse_solve<T>(pb, b, x);
  Level& lv = pb->L(l);
  Level& lc = pb->L(l - 1);
  const int extra = (lf - l) * prm.nu_inc;
  HHG_TRY(uzawa<T>(pb, lv, prm, prm.nu_pre + extra, x, b, vt<T>(lv)));
  HHG_TRY(residual<T>(pb, lv, x, b, vt<T>(lv)));
  HHG_TRY(restrict_to<T>(pb, l, vt<T>(lv), vb<T>(lc)));
  // the coarse correction starts from a zero guess (Algorithm 1)
  if (l - 1 > pb->desc.coarse_level)
    HHG_CUDA(launch_zero(vx<T>(lc), size_t(lc.nvec()) * sizeof(T), pb->stream));
  HHG_TRY(vcycle<T>(pb, lf, l - 1, prm, vx<T>(lc), vb<T>(lc)));
  HHG_TRY(prolong_add<T>(pb, l, vx<T>(lc), x));
  HHG_TRY(uzawa<T>(pb, lv, prm, prm.nu_post + extra, x, b, vt<T>(lv)));
  return HHG_OK;
}

// p <- p - (1^T M_L p / 1^T M_L 1) 1
int project_pressure(hhg_problem* pb, Level& lv, double* x) {
  const int64_t po = p_offset(lv);
  launch_reduce<double>(RED_WSUM, x + po, nullptr, lv.ml, lv.g.arr, pb->partials, pb->max_blocks, pb->scal, pb->stream);
  launch_sub_scalar_p<double>(lv.g, x + po, pb->scal, 1.0 / lv.ml_sum, pb->stream);
  HHG_CHECK_LAUNCH();
  return HHG_OK;
}

int fmg_interpolate(hhg_problem* pb, int l) {
  Level& f = pb->L(l);
  Level& c = pb->L(l - 1);
  launch_xpby<double>(c.x64, 1.0, c.W, c.tmp64, c.nvec(), pb->stream);
  HHG_CUDA(launch_zero(f.x64, size_t(f.nvec()) * 8, pb->stream));
  HHG_TRY(prolong_add<double>(pb, l, c.tmp64, f.x64, true));
  return HHG_OK;
}

int norms_of(hhg_problem* pb, Level& lv, int prec, const void* r, double* out2) {
  const int64_t po = p_offset(lv);
  if (prec == HHG_FP64) {
    const double* rr = static_cast<const double*>(r);
    launch_reduce<double>(RED_SQ, rr, nullptr, nullptr, po, pb->partials, pb->max_blocks, pb->scal + 1, pb->stream);
    launch_reduce<double>(RED_SQ, rr + po, nullptr, nullptr, lv.g.arr, pb->partials, pb->max_blocks, pb->scal + 2, pb->stream);
  } else {
    const float* rr = static_cast<const float*>(r);
    launch_reduce<float>(RED_SQ, rr, nullptr, nullptr, po, pb->partials, pb->max_blocks, pb->scal + 1, pb->stream);
    launch_reduce<float>(RED_SQ, rr + po, nullptr, nullptr, lv.g.arr, pb->partials, pb->max_blocks, pb->scal + 2, pb->stream);
  }
  HHG_CHECK_LAUNCH();
  double h[2];
  HHG_CUDA(cudaMemcpyAsync(h, pb->scal + 1, 16, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  out2[0] = std::sqrt(h[0]);
  out2[1] = std::sqrt(h[1]);
  return HHG_OK;
}

// dense LU with partial pivoting; returns the inverse of A (n x n, row-major)
bool invert(std::vector<double>& A, int n, std::vector<double>& inv) {
  std::vector<int> piv(n);
  for (int i = 0; i < n; ++i) piv[i] = i;
  for (int k = 0; k < n; ++k) {
    int p = k;
    double mx = std::fabs(A[size_t(k) * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (std::fabs(A[size_t(i) * n + k]) > mx) { mx = std::fabs(A[size_t(i) * n + k]); p = i; }
    if (mx == 0.0) return false;
    if (p != k) {
      for (int j = 0; j < n; ++j) std::swap(A[size_t(k) * n + j], A[size_t(p) * n + j]);
      std::swap(piv[k], piv[p]);
    }
    const double d = A[size_t(k) * n + k];
    for (int i = k + 1; i < n; ++i) {
      double f = A[size_t(i) * n + k] / d;
      A[size_t(i) * n + k] = f;
      if (f != 0.0)
        for (int j = k + 1; j < n; ++j) A[size_t(i) * n + j] -= f * A[size_t(k) * n + j];
    }
  }
  inv.assign(size_t(n) * n, 0.0);
  std::vector<double> col(n);
  for (int c = 0; c < n; ++c) {
    for (int i = 0; i < n; ++i) col[i] = piv[i] == c ? 1.0 : 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < i; ++j) col[i] -= A[size_t(i) * n + j] * col[j];
    for (int i = n - 1; i >= 0; --i) {
      for (int j = i + 1; j < n; ++j) col[i] -= A[size_t(i) * n + j] * col[j];
      col[i] /= A[size_t(i) * n + i];
    }
    for (int i = 0; i < n; ++i) inv[size_t(i) * n + c] = col[i];
  }
  return true;
}

int build_coarse(hhg_problem* pb) {
  Level& lv = pb->lv[0];
  const Geo& g = lv.g;
  std::vector<int64_t> idx;
  for (int c = 0; c < 3; ++c)
    for (int gg = 0; gg < pb->G; ++gg) {
      const int* o = kGroupOff[gg];
      for (int k = 0; k <= g.nz - o[2]; ++k)
        for (int j = 0; j <= g.ny - o[1]; ++j)
          for (int i = 0; i <= g.nx - o[0]; ++i) {
            int P[3] = {2 * i + o[0], 2 * j + o[1], 2 * k + o[2]};
            bool bnd = P[0] == 0 || P[1] == 0 || P[2] == 0 || P[0] == 2 * g.nx || P[1] == 2 * g.ny || P[2] == 2 * g.nz;
            if (!bnd) idx.push_back(int64_t(c * pb->G + gg) * g.arr + int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy);
          }
    }
  const int nu = int(idx.size());
  for (int k = 0; k <= g.nz; ++k)
    for (int j = 0; j <= g.ny; ++j)
      for (int i = 0; i <= g.nx; ++i)
        idx.push_back(p_offset(lv) + int64_t(i + 1) + int64_t(j + 1) * g.sx + int64_t(k + 1) * g.sy);
  const int n = int(idx.size());
  if (n != pb->ncoarse) return fail(HHG_EINVAL, "internal: coarse size mismatch");
  std::vector<double> host(size_t(lv.nvec()));
  std::vector<double> K(size_t(n + 1) * (n + 1), 0.0);
  const double one = 1.0;
  for (int jc = 0; jc < n; ++jc) {
    HHG_CUDA(cudaMemsetAsync(lv.tmp64, 0, size_t(lv.nvec()) * 8, pb->stream));
    HHG_CUDA(cudaMemcpyAsync(lv.tmp64 + idx[jc], &one, 8, cudaMemcpyHostToDevice, pb->stream));
    HHG_TRY(apply_op<double>(pb, lv, OP_FULL, MODE_SET, lv.tmp64, nullptr, lv.bw64));
    HHG_CUDA(cudaMemcpyAsync(host.data(), lv.bw64, host.size() * 8, cudaMemcpyDeviceToHost, pb->stream));
    HHG_CUDA(cudaStreamSynchronize(pb->stream));
    for (int r = 0; r < n; ++r) K[size_t(r) * (n + 1) + jc] = host[size_t(idx[r])];
  }
  // border with the lumped pressure mass (mean-zero constraint)
  std::vector<double> ml(size_t(g.arr));
  HHG_CUDA(cudaMemcpyAsync(ml.data(), lv.ml, ml.size() * 8, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  for (int r = nu; r < n; ++r) {
    const double m = ml[size_t(idx[r] - p_offset(lv))];
    K[size_t(r) * (n + 1) + n] = m;
    K[size_t(n) * (n + 1) + r] = m;
  }
  std::vector<double> inv;
  if (!invert(K, n + 1, inv)) return fail(HHG_EINVAL, "coarse system is singular (choose a finer coarse level)");
  std::vector<double> Z(size_t(n) * n);
  for (int r = 0; r < n; ++r)
    for (int c = 0; c < n; ++c) Z[size_t(r) * n + c] = inv[size_t(r) * (n + 1) + c];
  HHG_CUDA(cudaMemcpyAsync(pb->Z, Z.data(), Z.size() * 8, cudaMemcpyHostToDevice, pb->stream));
  HHG_CUDA(cudaMemcpyAsync(pb->cidx, idx.data(), idx.size() * 8, cudaMemcpyHostToDevice, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  return HHG_OK;
}

// ------------------------------------------------ learned coarse correction
// forward pass of the MLP on a batch X (B x n) into H1, H2 (B x h) and Y (B x n)
void nn_forward(hhg_problem* pb, const float* X, int B, float* H1, float* H2, float* Y) {
  const int n = pb->nn_n, h = pb->nn_h;
  const float* W1 = pb->nn_params;
  const float* b1 = W1 + int64_t(h) * n;
  const float* W2 = b1 + h;
  const float* b2 = W2 + int64_t(h) * h;
  const float* W3 = b2 + h;
  const float* b3 = W3 + int64_t(n) * h;
  nn_gemm(false, true, B, h, n, 1.f, X, n, W1, n, 0.f, H1, h, pb->stream);
  nn_bias_act(H1, b1, B, h, true, pb->stream);
  nn_gemm(false, true, B, h, h, 1.f, H1, h, W2, h, 0.f, H2, h, pb->stream);
  nn_bias_act(H2, b2, B, h, true, pb->stream);
  nn_gemm(false, true, B, n, h, 1.f, H2, h, W3, h, 0.f, Y, n, pb->stream);
  nn_bias_act(Y, b3, B, n, false, pb->stream);
}

// back-propagation of mean((Y - T)^2): gradients into nn_grads (same layout as the parameters)
void nn_backward(hhg_problem* pb, const float* X, const float* T, int B) {
  const int n = pb->nn_n, h = pb->nn_h;
  const float* W2 = pb->nn_params + int64_t(h) * n + h;
  const float* W3 = W2 + int64_t(h) * h + h;
  float* gW1 = pb->nn_grads;
  float* gb1 = gW1 + int64_t(h) * n;
  float* gW2 = gb1 + h;
  float* gb2 = gW2 + int64_t(h) * h;
  float* gW3 = gb2 + h;
  float* gb3 = gW3 + int64_t(n) * h;
  nn_mse(pb->nn_Y, T, int64_t(B) * n, 1.f / float(int64_t(B) * n), pb->nn_dY, pb->nn_part, pb->stream);
  nn_gemm(true, false, n, h, B, 1.f, pb->nn_dY, n, pb->nn_H2, h, 0.f, gW3, h, pb->stream);
  nn_colsum(pb->nn_dY, B, n, gb3, pb->stream);
  nn_gemm(false, false, B, h, n, 1.f, pb->nn_dY, n, W3, h, 0.f, pb->nn_dH2, h, pb->stream);
  nn_relu_back(pb->nn_dH2, pb->nn_H2, int64_t(B) * h, pb->stream);
  nn_gemm(true, false, h, h, B, 1.f, pb->nn_dH2, h, pb->nn_H1, h, 0.f, gW2, h, pb->stream);
  nn_colsum(pb->nn_dH2, B, h, gb2, pb->stream);
  nn_gemm(false, false, B, h, h, 1.f, pb->nn_dH2, h, W2, h, 0.f, pb->nn_dH1, h, pb->stream);
  nn_relu_back(pb->nn_dH1, pb->nn_H1, int64_t(B) * h, pb->stream);
  nn_gemm(true, false, h, n, B, 1.f, pb->nn_dH1, h, X, n, 0.f, gW1, n, pb->stream);
  nn_colsum(pb->nn_dH1, B, h, gb1, pb->stream);
}

int nn_setup(hhg_problem* pb) {
  const int n = pb->nn_n, h = pb->nn_h;
  Level& c = pb->lv[0];
  // FP32 copy of the coarse inverse and lumped masses of the pressure unknowns
  nn_to_float(pb->Z, pb->nn_Z, int64_t(n) * n, pb->stream);
  std::vector<int64_t> idx(n);
  HHG_CUDA(cudaMemcpyAsync(idx.data(), pb->cidx, size_t(n) * 8, cudaMemcpyDeviceToHost, pb->stream));
  std::vector<double> ml(size_t(c.g.arr));
  HHG_CUDA(cudaMemcpyAsync(ml.data(), c.ml, ml.size() * 8, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  const int64_t po = p_offset(c);
  int nu = 0;
  while (nu < n && idx[nu] < po) ++nu;
  std::vector<double> mlp(size_t(n - nu));
  for (int i = nu; i < n; ++i) mlp[size_t(i - nu)] = ml[size_t(idx[i] - po)];
  HHG_CUDA(cudaMemcpyAsync(pb->nn_mlp, mlp.data(), mlp.size() * 8, cudaMemcpyHostToDevice, pb->stream));
  // coordinates of the unknowns: array a = field * G + group (velocity) or 3G (pressure)
  std::vector<float> xyz(size_t(4) * n);
  const Geo& gc = c.g;
  for (int i = 0; i < n; ++i) {
    const int64_t a = idx[i] / gc.arr, site = idx[i] % gc.arr;
    const int64_t kk = site / gc.sy - 1, jj = (site % gc.sy) / gc.sx - 1, ii = site % gc.sx - 1;
    int field, grp;
    if (a < 3 * gc.G) { field = int(a / gc.G); grp = int(a % gc.G); }
    else { field = 3; grp = 0; }
    const int* o = kGroupOff[gc.G == 1 ? 0 : grp];
    xyz[size_t(4) * i + 0] = float((2 * ii + o[0]) * 0.5 * gc.h);
    xyz[size_t(4) * i + 1] = float((2 * jj + o[1]) * 0.5 * gc.h);
    xyz[size_t(4) * i + 2] = float((2 * kk + o[2]) * 0.5 * gc.h);
    xyz[size_t(4) * i + 3] = float(field);
  }
  HHG_CUDA(cudaMemcpyAsync(pb->nn_xyz, xyz.data(), xyz.size() * 4, cudaMemcpyHostToDevice, pb->stream));
  // He-style initial weights (fixed seed); Adam moments zero
  std::vector<float> P(size_t(pb->nn_P), 0.f);
  uint64_t st = 0x5EEDull;
  auto unif = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (double((st >> 11) & ((1ull << 53) - 1)) + 0.5) / double(1ull << 53);
  };
  auto gauss = [&]() { return std::sqrt(-2.0 * std::log(unif())) * std::cos(6.283185307179586 * unif()); };
  size_t o = 0;
  for (int64_t i = 0; i < int64_t(h) * n; ++i) P[o++] = float(gauss() * std::sqrt(2.0 / n));
  o += h;
  for (int64_t i = 0; i < int64_t(h) * h; ++i) P[o++] = float(gauss() * std::sqrt(2.0 / h));
  o += h;
  for (int64_t i = 0; i < int64_t(n) * h; ++i) P[o++] = float(gauss() * std::sqrt(1.0 / h));
  HHG_CUDA(cudaMemcpyAsync(pb->nn_params, P.data(), P.size() * 4, cudaMemcpyHostToDevice, pb->stream));
  HHG_CUDA(cudaMemsetAsync(pb->nn_m, 0, size_t(pb->nn_P) * 4, pb->stream));
  HHG_CUDA(cudaMemsetAsync(pb->nn_v, 0, size_t(pb->nn_P) * 4, pb->stream));
  HHG_CUDA(cudaMemsetAsync(pb->nn_counts, 0, 32, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  HHG_CHECK_LAUNCH();
  pb->nn_step = 0;
  return HHG_OK;
}

// learned coarse correction with the gate of hhg_coarse_nn_enable; x must be zero
template <class T>
int coarse_nn(hhg_problem* pb, const T* b, T* x) {
  const int n = pb->nn_n;
  nn_gather<T>(b, pb->cidx, n, pb->nn_xin, pb->nn_scal, pb->stream);
  nn_forward(pb, pb->nn_xin, 1, pb->nn_h1, pb->nn_h2, pb->nn_y);
  nn_scatter<T>(pb->nn_y, pb->cidx, n, pb->nn_scal, 1.0 / pb->nn_tscale, x, pb->stream);
  if (pb->nn_mode == 1) {
    Level& c = pb->lv[0];
    T* r = vt<T>(c);
    launch_apply<T>(c.g, c.op[OP_FULL], MODE_RES, x, b, r, 1.0, pb->stream);
    launch_reduce<T>(RED_SQ, r, nullptr, nullptr, c.nvec(), pb->partials, pb->max_blocks, pb->nn_scal + 1, pb->stream);
    nn_fallback<T>(pb->Z, n, pb->cidx, b, x, pb->nn_scal, pb->nn_theta, pb->nn_counts, pb->stream);
  }
  HHG_CHECK_LAUNCH();
  return HHG_OK;
}

}  // namespace

extern "C" int hhg_problem_bind(hhg_problem* pb, void* workspace, size_t bytes, void* stream) {
  if (!pb || !workspace) return fail(HHG_EINVAL, "null argument");
  if (bytes < pb->total) return fail(HHG_ENOMEM, "workspace smaller than hhg_problem_workspace_bytes");
  if (reinterpret_cast<uintptr_t>(workspace) % 256 != 0) return fail(HHG_EINVAL, "workspace must be 256-byte aligned");
  pb->ws = static_cast<char*>(workspace);
  pb->stream = static_cast<cudaStream_t>(stream);
  char* ws = pb->ws;
  // tables
  HHG_CUDA(cudaMemcpyAsync(ws + pb->o_tables, pb->tables.bytes.data(), pb->tables.bytes.size(), cudaMemcpyHostToDevice,
                           pb->stream));
  char* tb = ws + pb->o_tables;
  for (Level& lv : pb->lv) {
    for (int o = 0; o < OP_COUNT; ++o) {
      const OpOffsets& of = lv.opoff[o];
      OpDev& d = lv.op[o];
      d.rows = reinterpret_cast<const DRow*>(tb + of.rows);
      d.nrows = of.nrows;
      d.terms = reinterpret_cast<const DTerm*>(tb + of.terms);
      d.w64 = reinterpret_cast<const double*>(tb + of.w64);
      d.w32 = reinterpret_cast<const float*>(tb + of.w32);
      d.bterms = reinterpret_cast<const DTermB*>(tb + of.bterms);
      d.bw64 = reinterpret_cast<const double*>(tb + of.bw64);
      d.bw32 = reinterpret_cast<const float*>(tb + of.bw32);
    }
    lv.rhs = reinterpret_cast<double*>(ws + lv.o_rhs);
    lv.W = reinterpret_cast<double*>(ws + lv.o_W);
    lv.x64 = reinterpret_cast<double*>(ws + lv.o_x64);
    lv.tmp64 = reinterpret_cast<double*>(ws + lv.o_tmp64);
    lv.bw64 = reinterpret_cast<double*>(ws + lv.o_bw64);
    if (pb->desc.solve == HHG_SOLVE_MIXED) {
      lv.x32 = reinterpret_cast<float*>(ws + lv.o_x32);
      lv.b32 = reinterpret_cast<float*>(ws + lv.o_b32);
      lv.tmp32 = reinterpret_cast<float*>(ws + lv.o_tmp32);
    }
    lv.inv_mlhat = reinterpret_cast<double*>(ws + lv.o_invml);
    lv.ml = reinterpret_cast<double*>(ws + lv.o_ml);
  }
  auto xdev = [&](const XferOffsets& xo) {
    XferDev X;
    X.order = xo.order; X.nclass = xo.nclass; X.ngroups = xo.ngroups;
    X.pcls_start = reinterpret_cast<const int*>(tb + xo.pstart);
    X.pterms = reinterpret_cast<const DXTerm*>(tb + xo.pterms);
    X.pw64 = reinterpret_cast<const double*>(tb + xo.pw64);
    X.pw32 = reinterpret_cast<const float*>(tb + xo.pw32);
    X.rg_start = reinterpret_cast<const int*>(tb + xo.rstart);
    X.rterms = reinterpret_cast<const DXTerm*>(tb + xo.rterms);
    X.rw64 = reinterpret_cast<const double*>(tb + xo.rw64);
    X.rw32 = reinterpret_cast<const float*>(tb + xo.rw32);
    X.rmax = xo.rmax;
    return X;
  };
  pb->xv = xdev(pb->xoff_v);
  pb->xp = xdev(pb->xoff_p);
  pb->Z = reinterpret_cast<double*>(ws + pb->o_Z);
  pb->cidx = reinterpret_cast<int64_t*>(ws + pb->o_idx);
  pb->partials = reinterpret_cast<double*>(ws + pb->o_part);
  pb->scal = reinterpret_cast<double*>(ws + pb->o_scal);
  if (pb->nn_h > 0) {
    const int n = pb->nn_n, h = pb->nn_h;
    const int64_t B = pb->nn_B;
    float* f = reinterpret_cast<float*>(ws + pb->o_nn);
    auto take = [&](int64_t cnt) { float* r = f; f += cnt; return r; };
    pb->nn_params = take(pb->nn_P); pb->nn_grads = take(pb->nn_P); pb->nn_m = take(pb->nn_P); pb->nn_v = take(pb->nn_P);
    pb->nn_Z = take(int64_t(n) * n);
    pb->nn_X = take(int64_t(pb->nn_S) * n); pb->nn_T = take(int64_t(pb->nn_S) * n);
    pb->nn_H1 = take(B * h); pb->nn_H2 = take(B * h); pb->nn_dH1 = take(B * h); pb->nn_dH2 = take(B * h);
    pb->nn_Y = take(B * n); pb->nn_dY = take(B * n);
    pb->nn_xin = take(n); pb->nn_y = take(n); pb->nn_h1 = take(h); pb->nn_h2 = take(h);
    f = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(f) + 15) / 16 * 16);
    pb->nn_xyz = take(4 * int64_t(n));
    char* c = reinterpret_cast<char*>(ws + pb->o_nn) + align256(size_t(f - reinterpret_cast<float*>(ws + pb->o_nn)) * 4);
    pb->nn_mlp = reinterpret_cast<double*>(c); c += align256(size_t(n) * 8);
    pb->nn_scal = reinterpret_cast<double*>(c); c += align256(64 * 8);
    pb->nn_part = reinterpret_cast<double*>(c); c += align256(1024 * 8);
    pb->nn_counts = reinterpret_cast<unsigned long long*>(c);
  }
  // zero all vectors (halo and padding stay zero for the lifetime of the problem)
  HHG_CUDA(cudaMemsetAsync(ws + pb->lv[0].o_rhs, 0, pb->o_Z - pb->lv[0].o_rhs, pb->stream));
  pb->bound = true;
  // viscosity row scales exp(+-nu_a h k) of every level (after the memset above)
  for (Level& lv : pb->lv) {
    double* esc = reinterpret_cast<double*>(ws + lv.o_esc);
    std::vector<double> tab(size_t(2 * (lv.g.nz + 1)));
    for (int k = 0; k <= lv.g.nz; ++k) {
      tab[size_t(k)] = std::exp(lv.g.nu_ah * k);
      tab[size_t(lv.g.nz + 1 + k)] = std::exp(-lv.g.nu_ah * k);
    }
    HHG_CUDA(cudaMemcpyAsync(esc, tab.data(), tab.size() * 8, cudaMemcpyHostToDevice, pb->stream));
    HHG_CUDA(cudaStreamSynchronize(pb->stream));
    lv.g.esc = esc;
    lv.g.eisc = esc + lv.g.nz + 1;
  }
  // lumped masses: M_L 1 (projection weights) and M_L(1/nu) (S_hat)
  for (Level& lv : pb->lv) {
    const int64_t po = p_offset(lv);
    // ones on all pressure nodes (in tmp64)
    std::vector<double> ones(size_t(lv.nvec()), 0.0);
    for_each_pressure_node(lv.g, [&](int64_t, int64_t site) { ones[size_t(po + site)] = 1.0; });
    HHG_CUDA(cudaMemcpyAsync(lv.tmp64, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, pb->stream));
    HHG_TRY(apply_op<double>(pb, lv, OP_ML, MODE_SET, lv.tmp64, nullptr, lv.bw64));
    HHG_CUDA(cudaMemcpyAsync(lv.ml, lv.bw64 + po, size_t(lv.g.arr) * 8, cudaMemcpyDeviceToDevice, pb->stream));
    HHG_TRY(apply_op<double>(pb, lv, OP_MLHAT, MODE_SET, lv.tmp64, nullptr, lv.bw64));
    launch_inv(lv.bw64 + po, lv.inv_mlhat, lv.g.arr, pb->stream);
    launch_reduce<double>(RED_SUM, lv.ml, nullptr, nullptr, lv.g.arr, pb->partials, pb->max_blocks, pb->scal, pb->stream);
    HHG_CHECK_LAUNCH();
    HHG_CUDA(cudaMemcpyAsync(&lv.ml_sum, pb->scal, 8, cudaMemcpyDeviceToHost, pb->stream));
    HHG_CUDA(cudaStreamSynchronize(pb->stream));
    HHG_CUDA(cudaMemsetAsync(lv.tmp64, 0, size_t(lv.nvec()) * 8, pb->stream));
    HHG_CUDA(cudaMemsetAsync(lv.bw64, 0, size_t(lv.nvec()) * 8, pb->stream));
  }
  HHG_TRY(build_coarse(pb));
  if (pb->nn_h > 0) HHG_TRY(nn_setup(pb));
  stream_init<float>();
  stream_init<double>();
  for (Level& lv : pb->lv) {
    HHG_TRY(default_resident(pb, lv, HHG_FP64));
    HHG_TRY(default_resident(pb, lv, HHG_FP32));
  }
  Level& c = pb->lv[0];
  HHG_CUDA(cudaMemsetAsync(c.tmp64, 0, size_t(c.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaMemsetAsync(c.bw64, 0, size_t(c.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  return HHG_OK;
}

// ------------------------------------------------------------------- rhs
namespace {
// enqueues the assembly of one level's right-hand side on the problem's
// stream (the caller synchronises before the host buffers are reused)
int enqueue_rhs(hhg_problem* pb, int level, const double* f_nodal, const double* w_nodal) {
  HHG_TRY(check_level(pb, level));
  if (!f_nodal || !w_nodal) return fail(HHG_EINVAL, "null nodal data");
  Level& lv = pb->L(level);
  const Geo& g = lv.g;
  const int64_t nvn = velocity_nodes(g), npn = pressure_nodes(g);
  // nodal data to the layout: F at every velocity node, W at the boundary ones
  HHG_CUDA(cudaMemsetAsync(lv.tmp64, 0, size_t(lv.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaMemsetAsync(lv.W, 0, size_t(lv.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaMemcpyAsync(lv.bw64, f_nodal, size_t(3 * nvn) * 8, cudaMemcpyHostToDevice, pb->stream));
  launch_canon_scatter<double>(g, lv.bw64, lv.tmp64, nvn, npn, false, false, pb->stream);
  HHG_CUDA(cudaMemcpyAsync(lv.bw64, w_nodal, size_t(3 * nvn) * 8, cudaMemcpyHostToDevice, pb->stream));
  launch_canon_scatter<double>(g, lv.bw64, lv.W, nvn, npn, false, true, pb->stream);
  HHG_CHECK_LAUNCH();
  HHG_CUDA(cudaMemsetAsync(lv.rhs, 0, size_t(lv.nvec()) * 8, pb->stream));
  // f = M f_h - A w_h (interior velocity rows); w_h is non-zero only on
  // boundary nodes, so A w_h and B w_h are evaluated on the shell of rows
  // within one site of the box's faces (the others read no boundary node)
  HHG_TRY(apply_op<double>(pb, lv, OP_MVINT, MODE_SET, lv.tmp64, nullptr, lv.rhs));
  launch_apply_shell<double>(lv.g, lv.op[OP_A], MODE_ADD, lv.W, nullptr, lv.rhs, -1.0, pb->stream);
  // g = -B w_h (+ PSPG load), projected to sum zero
  launch_apply_shell<double>(lv.g, lv.op[OP_B], MODE_ADD, lv.W, nullptr, lv.rhs, -1.0, pb->stream);
  HHG_CHECK_LAUNCH();
  if (pb->ov == 1 && pb->desc.pspg_rhs) HHG_TRY(apply_op<double>(pb, lv, OP_LOAD, MODE_ADD, lv.tmp64, nullptr, lv.rhs, 1.0));
  const int64_t po = p_offset(lv);
  // the mean's partial sums in the level's own scratch vector where it holds
  // them (so that a finest-level assembly may overlap solver stages, which use
  // the problem's reduction buffers)
  const bool own = lv.nvec() >= int64_t(pb->max_blocks) + 8;
  double* part = own ? lv.bw64 : pb->partials;
  double* sum = own ? lv.bw64 + pb->max_blocks : pb->scal;
  launch_reduce<double>(RED_SUM, lv.rhs + po, nullptr, nullptr, g.arr, part, pb->max_blocks, sum, pb->stream);
  launch_sub_scalar_p<double>(g, lv.rhs + po, sum, 1.0 / double((g.nx + 1) * int64_t(g.ny + 1) * (g.nz + 1)), pb->stream);
  HHG_CHECK_LAUNCH();
  HHG_CUDA(cudaMemsetAsync(lv.tmp64, 0, size_t(lv.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaMemsetAsync(lv.bw64, 0, size_t(lv.nvec()) * 8, pb->stream));
  lv.has_rhs = true;
  return HHG_OK;
}
}  // namespace

// arguments of one level's rhs, checked before anything is queued
static int check_rhs_args(hhg_problem* pb, int level, const double* f_nodal, const double* w_nodal) {
  HHG_TRY(check_level(pb, level));
  if (!f_nodal || !w_nodal) return fail(HHG_EINVAL, "null nodal data");
  return HHG_OK;
}

// a failure after work was queued: wait for the queued copies, so that the
// caller's host buffers are free when the error is returned
static int fail_after_queue(hhg_problem* pb, int rc) {
  cudaStreamSynchronize(pb->stream);
  return rc;
}

extern "C" int hhg_set_rhs(hhg_problem* pb, int level, const double* f_nodal, const double* w_nodal) {
  HHG_TRY(check_rhs_args(pb, level, f_nodal, w_nodal));
  const int rc = enqueue_rhs(pb, level, f_nodal, w_nodal);
  if (rc != HHG_OK) return fail_after_queue(pb, rc);
  HHG_CUDA(cudaStreamSynchronize(pb->stream));    // the host buffers may be reused on return
  return HHG_OK;
}

extern "C" int hhg_set_rhs_levels(hhg_problem* pb, int l0, int l1, const double* const* f_nodal,
                                  const double* const* w_nodal) {
  if (!pb) return fail(HHG_EINVAL, "null problem");
  if (!f_nodal || !w_nodal || l1 < l0) return fail(HHG_EINVAL, "invalid level range or null pointer arrays");
  // every level and pointer is checked first: an invalid call changes nothing
  for (int l = l0; l <= l1; ++l) HHG_TRY(check_rhs_args(pb, l, f_nodal[l - l0], w_nodal[l - l0]));
  for (int l = l0; l <= l1; ++l) {
    const int rc = enqueue_rhs(pb, l, f_nodal[l - l0], w_nodal[l - l0]);
    if (rc != HHG_OK) return fail_after_queue(pb, rc);
  }
  HHG_CUDA(cudaStreamSynchronize(pb->stream));    // one wait for all levels
  return HHG_OK;
}

extern "C" int hhg_level_vector(hhg_problem* pb, int level, int which, void** dev) {
  HHG_TRY(check_level(pb, level));
  if (!dev) return fail(HHG_EINVAL, "null output");
  Level& lv = pb->L(level);
  if (which == 0) *dev = lv.rhs;
  else if (which == 1) *dev = lv.W;
  else if (which == 2) *dev = lv.x64;
  else return fail(HHG_EINVAL, "unknown level vector");
  return HHG_OK;
}

// ---------------------------------------------------------- public steps
namespace {
int check_params(const hhg_params* prm) {
  if (!prm) return fail(HHG_EINVAL, "null params");
  if (prm->nu_pre < 0 || prm->nu_post < 0 || prm->nu_inc < 0 || prm->kappa < 1 || prm->xi < 1 ||
      (prm->ahat != HHG_AHAT_F && prm->ahat != HHG_AHAT_S) || !(prm->omega_inv > 0))
    return fail(HHG_EINVAL, "invalid FMG parameters");
  return HHG_OK;
}
}  // namespace

extern "C" int hhg_apply(hhg_problem* pb, int level, int op, int prec, const void* x, void* y) {
  HHG_TRY(check_level(pb, level, op == HHG_OP_MASS));
  HHG_TRY(check_prec(pb, prec));
  if (!x || !y) return fail(HHG_EINVAL, "null vector");
  int id;
  switch (op) {
    case HHG_OP_FULL: id = OP_FULL; break;
    case HHG_OP_A: id = OP_A; break;
    case HHG_OP_BT: id = OP_BT; break;
    case HHG_OP_B: id = OP_B; break;
    case HHG_OP_C: id = OP_C; break;
    case HHG_OP_MASS: id = OP_MASS; break;
    default: return fail(HHG_EINVAL, "unknown operator");
  }
  Level& lv = pb->L(level);
  const size_t es = prec == HHG_FP64 ? 8 : 4;
  if (id != OP_FULL && id != OP_MASS) HHG_CUDA(cudaMemsetAsync(y, 0, size_t(lv.nvec()) * es, pb->stream));
  if (id == OP_C && pb->ov == 2) return HHG_OK;              // C = 0 for Taylor-Hood
  if (prec == HHG_FP64)
    return apply_op<double>(pb, lv, id, MODE_SET, static_cast<const double*>(x), nullptr, static_cast<double*>(y));
  return apply_op<float>(pb, lv, id, MODE_SET, static_cast<const float*>(x), nullptr, static_cast<float*>(y));
}

extern "C" int hhg_residual(hhg_problem* pb, int level, int prec, const void* x, const void* b, void* r, double* norms) {
  HHG_TRY(check_level(pb, level));
  HHG_TRY(check_prec(pb, prec));
  if (!x || !b || !r) return fail(HHG_EINVAL, "null vector");
  Level& lv = pb->L(level);
  if (prec == HHG_FP64)
    HHG_TRY(residual<double>(pb, lv, static_cast<const double*>(x), static_cast<const double*>(b), static_cast<double*>(r)));
  else
    HHG_TRY(residual<float>(pb, lv, static_cast<const float*>(x), static_cast<const float*>(b), static_cast<float*>(r)));
  if (norms) HHG_TRY(norms_of(pb, lv, prec, r, norms));
  return HHG_OK;
}

extern "C" int hhg_refinement_residual(hhg_problem* pb, int level, const double* x, const double* b, float* r) {
  HHG_TRY(check_level(pb, level));
  if (pb->desc.solve != HHG_SOLVE_MIXED) return fail(HHG_EINVAL, "the refinement residual needs a mixed-precision problem");
  if (!x || !b || !r) return fail(HHG_EINVAL, "null vector");
  if (reinterpret_cast<uintptr_t>(x) & 15) return fail(HHG_EINVAL, "x must be 16-byte aligned");
  Level& lv = pb->L(level);
  return refinement_residual(pb, lv, x, b, r);
}

extern "C" int hhg_smooth(hhg_problem* pb, int level, const hhg_params* prm, int sweeps, int prec, void* x, const void* b) {
  HHG_TRY(check_level(pb, level));
  HHG_TRY(check_params(prm));
  HHG_TRY(check_prec(pb, prec));
  if (!x || !b || sweeps < 0) return fail(HHG_EINVAL, "bad smoother arguments");
  Level& lv = pb->L(level);
  if (prec == HHG_FP64)
    return uzawa<double>(pb, lv, *prm, sweeps, static_cast<double*>(x), static_cast<const double*>(b), lv.tmp64);
  return uzawa<float>(pb, lv, *prm, sweeps, static_cast<float*>(x), static_cast<const float*>(b), lv.tmp32);
}

extern "C" int hhg_restrict(hhg_problem* pb, int level, int prec, const void* r_fine, void* r_coarse) {
  HHG_TRY(check_level(pb, level));
  HHG_TRY(check_prec(pb, prec));
  if (level <= pb->desc.coarse_level) return fail(HHG_EINVAL, "no coarser level");
  if (!r_fine || !r_coarse) return fail(HHG_EINVAL, "null vector");
  if (prec == HHG_FP64) return restrict_to<double>(pb, level, static_cast<const double*>(r_fine), static_cast<double*>(r_coarse));
  return restrict_to<float>(pb, level, static_cast<const float*>(r_fine), static_cast<float*>(r_coarse));
}

extern "C" int hhg_prolongate_add(hhg_problem* pb, int level, int prec, const void* x_coarse, void* x_fine) {
  HHG_TRY(check_level(pb, level));
  HHG_TRY(check_prec(pb, prec));
  if (level <= pb->desc.coarse_level) return fail(HHG_EINVAL, "no coarser level");
  if (!x_coarse || !x_fine) return fail(HHG_EINVAL, "null vector");
  if (prec == HHG_FP64) return prolong_add<double>(pb, level, static_cast<const double*>(x_coarse), static_cast<double*>(x_fine));
  return prolong_add<float>(pb, level, static_cast<const float*>(x_coarse), static_cast<float*>(x_fine));
}

extern "C" int hhg_coarse_solve(hhg_problem* pb, int prec, const void* b, void* x) {
  HHG_TRY(check_level(pb, pb ? pb->desc.coarse_level : 0));
  HHG_TRY(check_prec(pb, prec));
  if (!b || !x) return fail(HHG_EINVAL, "null vector");
  if (prec == HHG_FP64) return coarse_solve<double>(pb, static_cast<const double*>(b), static_cast<double*>(x));
  return coarse_solve<float>(pb, static_cast<const float*>(b), static_cast<float*>(x));
}

extern "C" int hhg_vcycle(hhg_problem* pb, int level, const hhg_params* prm, int prec, void* x, const void* b) {
  HHG_TRY(check_level(pb, level));
  HHG_TRY(check_params(prm));
  HHG_TRY(check_prec(pb, prec));
  if (!x || !b) return fail(HHG_EINVAL, "null vector");
  if (prec == HHG_FP64) return vcycle<double>(pb, level, level, *prm, static_cast<double*>(x), static_cast<const double*>(b));
  return vcycle<float>(pb, level, level, *prm, static_cast<float*>(x), static_cast<const float*>(b));
}

namespace {
double model_wu(const hhg_problem* pb, const hhg_params& p) {
  const Costs c = block_costs(pb->ov);
  const double wa = p.ahat == HHG_AHAT_S ? 2 * c.A : c.A;
  const double wp = p.xi * wa + 2 * c.B + c.C;
  const double wv = (p.nu_pre + p.nu_post) * wp + 1.0;
  return 8.0 * p.kappa / 7.0 * (8.0 / 7.0 * wv + 16.0 / 49.0 * p.nu_inc * wp);
}
}  // namespace

namespace {
// the kernel sequence of one FMG solve (Algorithm 1), or of its stages
// first..last (stage lc: the coarse solve; stage l > lc: the FMG
// interpolation to level l and its kappa cycles); no host synchronisation
int fmg_core(hhg_problem* pb, const hhg_params* prm, int first = -1, int last = -1) {
  const int lc = pb->desc.coarse_level;
  if (first < 0) first = lc;
  if (last < 0) last = pb->desc.L;
  if (first == lc) {
    pb->wu_counted = 0.0;
    Level& c = pb->L(lc);
    HHG_TRY(coarse_solve<double>(pb, c.rhs, c.x64));
    HHG_TRY(project_pressure(pb, c, c.x64));
  }
  for (int l = std::max(first, lc + 1); l <= last; ++l) {
    Level& lv = pb->L(l);
    HHG_TRY(fmg_interpolate(pb, l));
    for (int kk = 0; kk < prm->kappa; ++kk) {
      if (pb->desc.solve == HHG_SOLVE_FP64) {
        HHG_TRY(vcycle<double>(pb, l, l, *prm, lv.x64, lv.rhs));
      } else {
        // iterative refinement: residual of the FP64 iterate (FP64, or
        // double-float into FP32), FP32 V-cycle on the defect, FP64 update
        HHG_TRY(refinement_residual(pb, lv, lv.x64, lv.rhs, lv.b32));
        HHG_CUDA(launch_zero(lv.x32, size_t(lv.nvec()) * 4, pb->stream));
        HHG_TRY(vcycle<float>(pb, l, l, *prm, lv.x32, lv.b32));
        launch_add_f2d(lv.x32, lv.x64, lv.nvec(), pb->stream);
        HHG_CHECK_LAUNCH();
      }
      HHG_TRY(project_pressure(pb, lv, lv.x64));
    }
  }
  return HHG_OK;
}

bool capturable(cudaStream_t s) {
  return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread;
}
}  // namespace

extern "C" int hhg_set_refinement_residual(hhg_problem* pb, int kind) {
  if (!pb) return fail(HHG_EINVAL, "null problem");
  if (kind != HHG_REFINE_FP64 && kind != HHG_REFINE_DF32)
    return fail(HHG_EINVAL, "kind must be HHG_REFINE_FP64 or HHG_REFINE_DF32");
  if (kind == HHG_REFINE_DF32 && !df_supported(pb->desc.disc, pb->desc.nu_a != 0.0 ? 1 : 0))
    return fail(HHG_EINVAL, "the double-float residual does not cover this operator");
  if (pb->refine != kind) {
    for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
    pb->graphs.clear();
  }
  pb->refine = kind;
  return HHG_OK;
}

extern "C" int hhg_get_refinement_residual(hhg_problem* pb, int* kind) {
  if (!pb || !kind) return fail(HHG_EINVAL, "null argument");
  *kind = pb->refine == HHG_REFINE_DF32 && df_supported(pb->desc.disc, pb->desc.nu_a != 0.0 ? 1 : 0)
              ? HHG_REFINE_DF32
              : HHG_REFINE_FP64;
  return HHG_OK;
}

extern "C" int hhg_set_graph_mode(hhg_problem* pb, int on) {
  if (!pb) return fail(HHG_EINVAL, "null problem");
  pb->use_graphs = on != 0;
  return HHG_OK;
}

extern "C" int hhg_set_level_smoother(hhg_problem* pb, int level, int prec, int ctas, int threads) {
  HHG_TRY(check_level(pb, level));
  if (prec != HHG_FP64 && prec != HHG_FP32) return fail(HHG_EINVAL, "prec must be HHG_FP64 or HHG_FP32");
  HHG_TRY(set_resident(pb, pb->L(level), prec, ctas, threads == 0 ? kResidentThreads : threads));
  for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
  pb->graphs.clear();
  return HHG_OK;
}

extern "C" int hhg_get_level_smoother(hhg_problem* pb, int level, int prec, int* ctas, int* threads) {
  HHG_TRY(check_level(pb, level));
  if (prec != HHG_FP64 && prec != HHG_FP32) return fail(HHG_EINVAL, "prec must be HHG_FP64 or HHG_FP32");
  if (!ctas || !threads) return fail(HHG_EINVAL, "null argument");
  *ctas = pb->L(level).rctas[prec];
  *threads = pb->L(level).rthreads[prec];
  return HHG_OK;
}

extern "C" int hhg_set_launch_shape(hhg_problem* pb, int level, int row_threads, int row_kplanes, int gs_threads,
                                    int row_tile, int row_sites, int gs_lanes) {
  HHG_TRY(check_level(pb, level));
  auto ok_threads = [](int t) { return t == 64 || t == 128 || t == 256; };
  if (!ok_threads(row_threads) || !ok_threads(gs_threads) || row_kplanes < 1 || row_kplanes > 64 ||
      (row_tile != 0 && row_tile != 1 && !ok_threads(row_tile)) ||
      (row_sites != 1 && row_sites != 4 && !(row_sites == 2 && row_tile != 0)) ||
      (gs_lanes != 1 && gs_lanes != 2 && gs_lanes != 4))
    return fail(HHG_EINVAL, "invalid launch shape");
  Shape& sh = pb->L(level).shape;
  sh.row_threads = row_threads;
  sh.row_kplanes = row_kplanes;
  sh.gs_threads = gs_threads;
  const int st = row_tile == 1 ? 128 : row_tile;
  for (int o = 0; o < 3; ++o) {
    sh.st_threads[o] = sh.st64_threads[o] = st;
    sh.st_sites[o] = row_sites == 2 ? 2 : 4;
  }
  sh.row_sites = row_sites == 2 ? 4 : row_sites;
  sh.row_sites64 = row_sites;
  sh.gs_lanes = gs_lanes;
  sh.gs_lanes0 = gs_lanes;
  sh.gs_threads0 = 0;
  sh.bt_threads = sh.bt_kplanes = sh.bt_sites = 0;
  sh.bc_threads = sh.bc_kplanes = sh.bc_sites = 0;
  for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
  pb->graphs.clear();
  return HHG_OK;
}

extern "C" int hhg_set_level_sweep_order(hhg_problem* pb, int level, int order) {
  HHG_TRY(check_level(pb, level));
  if (order != 0 && order != 1) return fail(HHG_EINVAL, "order must be 0 or 1");
  pb->L(level).shape.gs_comp_major = order;
  for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
  pb->graphs.clear();
  return HHG_OK;
}

extern "C" int hhg_get_level_sweep_order(hhg_problem* pb, int level, int* order) {
  HHG_TRY(check_level(pb, level));
  if (!order) return fail(HHG_EINVAL, "null argument");
  *order = pb->L(level).shape.gs_comp_major;
  return HHG_OK;
}

extern "C" int hhg_get_launch_shape(hhg_problem* pb, int level, int* shape6) {
  HHG_TRY(check_level(pb, level));
  if (!shape6) return fail(HHG_EINVAL, "null argument");
  const Shape& sh = pb->L(level).shape;
  shape6[0] = sh.row_threads; shape6[1] = sh.row_kplanes; shape6[2] = sh.gs_threads; shape6[3] = sh.st_threads[0];
  shape6[4] = sh.st_threads[0] && sh.st_sites[0] == 2 ? 2 : sh.row_sites; shape6[5] = sh.gs_lanes;
  return HHG_OK;
}

extern "C" int hhg_set_small_level_mode(hhg_problem* pb, int on) {
  if (!pb) return fail(HHG_EINVAL, "null problem");
  pb->use_cluster = on != 0;
  for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
  pb->graphs.clear();
  return HHG_OK;
}

namespace {
// stages first..last of the FMG on pb->stream: recorded once per parameter
// tuple and part as a CUDA graph and replayed (or launched directly when
// graphs are off or the stream cannot be captured); adds the kernel count
int run_stages(hhg_problem* pb, const hhg_params* prm, int part, int first, int last, int64_t* kernels) {
  if (pb->use_graphs && capturable(pb->stream)) {
    auto key = std::make_tuple(prm->nu_pre, prm->nu_post, prm->nu_inc, prm->kappa, prm->ahat, prm->xi, prm->omega_inv,
                               part);
    auto it = pb->graphs.find(key);
    if (it == pb->graphs.end()) {
      const int64_t l0 = g_launches;
      const double wu0 = first == pb->desc.coarse_level ? 0.0 : pb->wu_counted;   // fmg_core restarts the count
      HHG_CUDA(cudaStreamBeginCapture(pb->stream, cudaStreamCaptureModeThreadLocal));
      int rc = fmg_core(pb, prm, first, last);
      cudaGraph_t graph = nullptr;
      cudaError_t ec = cudaStreamEndCapture(pb->stream, &graph);
      if (rc != HHG_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
      if (ec != cudaSuccess) return fail(HHG_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ec));
      cudaGraphExec_t exec;
      cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ei != cudaSuccess) return fail(HHG_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ei));
      it = pb->graphs.emplace(key, hhg_problem::Graph{exec, g_launches - l0, pb->wu_counted - wu0}).first;
      pb->wu_counted = wu0;       // the capture counted the stages; the replay below counts them once
    }
    HHG_CUDA(cudaGraphLaunch(it->second.exec, pb->stream));
    *kernels += it->second.kernels;
    pb->wu_counted = (first == pb->desc.coarse_level ? 0.0 : pb->wu_counted) + it->second.wu;
  } else {
    const int64_t l0 = g_launches;
    HHG_TRY(fmg_core(pb, prm, first, last));
    *kernels += g_launches - l0;
  }
  return HHG_OK;
}

int fill_stats(hhg_problem* pb, const hhg_params* prm, int64_t kernels, hhg_stats* stats) {
  Level& top = pb->L(pb->desc.L);
  stats->wu_model = model_wu(pb, *prm);
  stats->wu_counted = pb->wu_counted;
  HHG_TRY(residual<double>(pb, top, top.x64, top.rhs, top.tmp64));
  double nr[2];
  HHG_TRY(norms_of(pb, top, HHG_FP64, top.tmp64, nr));
  stats->res_u = nr[0];
  stats->res_p = nr[1];
  stats->kernel_launches = kernels;
  if (!std::isfinite(nr[0]) || !std::isfinite(nr[1])) return fail(HHG_EDIVERGED, "FMG produced a non-finite residual");
  return HHG_OK;
}
}  // namespace

extern "C" int hhg_fmg_solve(hhg_problem* pb, const hhg_params* prm, void* x_out, hhg_stats* stats) {
  HHG_TRY(check_level(pb, pb ? pb->desc.L : 0));
  HHG_TRY(check_params(prm));
  for (int l = pb->desc.coarse_level; l <= pb->desc.L; ++l)
    if (!pb->L(l).has_rhs) return fail(HHG_ESTATE, "hhg_set_rhs missing on a level");
  int64_t kernels = 0;
  HHG_TRY(run_stages(pb, prm, 0, pb->desc.coarse_level, pb->desc.L, &kernels));
  Level& top = pb->L(pb->desc.L);
  if (x_out) HHG_CUDA(cudaMemcpyAsync(x_out, top.x64, size_t(top.nvec()) * 8, cudaMemcpyDeviceToDevice, pb->stream));
  if (stats) HHG_TRY(fill_stats(pb, prm, kernels, stats));
  return HHG_OK;
}

extern "C" int hhg_fmg_solve_host(hhg_problem* pb, const hhg_params* prm, const double* const* f_nodal,
                                  const double* const* w_nodal, double* x_host, hhg_stats* stats) {
  if (!pb) return fail(HHG_EINVAL, "null problem");
  HHG_TRY(check_params(prm));
  if (!f_nodal || !w_nodal) return fail(HHG_EINVAL, "null pointer arrays");
  const int lc = pb->desc.coarse_level, L = pb->desc.L;
  for (int l = lc; l <= L; ++l) HHG_TRY(check_rhs_args(pb, l, f_nodal[l - lc], w_nodal[l - lc]));
  if (!pb->aux) {
    int least = 0, greatest = 0;
    HHG_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    HHG_CUDA(cudaStreamCreateWithFlags(&pb->aux, cudaStreamNonBlocking));
    HHG_CUDA(cudaStreamCreateWithPriority(&pb->hp, cudaStreamNonBlocking, greatest));
    for (cudaEvent_t* e : {&pb->ev_start, &pb->ev_coarse, &pb->ev_fine, &pb->ev_done})
      HHG_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  }
  cudaStream_t main = pb->stream;
  // the finest level's assembly may run beside the stages below it when its
  // scratch holds the reduction and the stages replay as graphs
  const bool overlap = L > lc && pb->use_graphs && capturable(main) &&
                       pb->L(L).nvec() >= int64_t(pb->max_blocks) + 8;
  // right-hand sides on the second stream, after the work already queued on
  // the problem's stream (which may still read the previous ones)
  HHG_CUDA(cudaEventRecord(pb->ev_start, main));
  HHG_CUDA(cudaStreamWaitEvent(pb->aux, pb->ev_start, 0));
  pb->stream = pb->aux;
  int rc = HHG_OK;
  for (int l = lc; l < L && rc == HHG_OK; ++l) rc = enqueue_rhs(pb, l, f_nodal[l - lc], w_nodal[l - lc]);
  if (rc == HHG_OK) rc = cudaEventRecord(pb->ev_coarse, pb->aux) == cudaSuccess ? HHG_OK : fail(HHG_ECUDA, "event record");
  if (rc == HHG_OK) rc = enqueue_rhs(pb, L, f_nodal[L - lc], w_nodal[L - lc]);
  if (rc == HHG_OK) rc = cudaEventRecord(pb->ev_fine, pb->aux) == cudaSuccess ? HHG_OK : fail(HHG_ECUDA, "event record");
  pb->stream = main;
  if (rc != HHG_OK) {
    cudaStreamSynchronize(pb->aux);
    return rc;
  }
  // the FMG: the stages below L once the coarse right-hand sides are in,
  // stage L once the finest one is
  int64_t kernels = 0;
  if (overlap) {
    // the stages on a stream of the highest priority, so that their short
    // launches go first while the finest level's assembly holds the SMs
    HHG_CUDA(cudaStreamWaitEvent(pb->hp, pb->ev_start, 0));
    HHG_CUDA(cudaStreamWaitEvent(pb->hp, pb->ev_coarse, 0));
    pb->stream = pb->hp;
    rc = run_stages(pb, prm, 1, lc, L - 1, &kernels);
    if (rc == HHG_OK) rc = cudaStreamWaitEvent(pb->hp, pb->ev_fine, 0) == cudaSuccess ? HHG_OK : fail(HHG_ECUDA, "wait");
    if (rc == HHG_OK) rc = run_stages(pb, prm, 2, L, L, &kernels);
    pb->stream = main;
    if (rc == HHG_OK) rc = cudaEventRecord(pb->ev_done, pb->hp) == cudaSuccess ? HHG_OK : fail(HHG_ECUDA, "event record");
    if (rc == HHG_OK) rc = cudaStreamWaitEvent(main, pb->ev_done, 0) == cudaSuccess ? HHG_OK : fail(HHG_ECUDA, "wait");
  } else {
    HHG_CUDA(cudaStreamWaitEvent(main, pb->ev_fine, 0));
    rc = run_stages(pb, prm, 0, lc, L, &kernels);
  }
  // the solution in canonical order to the host
  Level& top = pb->L(L);
  if (rc == HHG_OK && x_host) {
    const int64_t nvn = velocity_nodes(top.g), npn = pressure_nodes(top.g);
    launch_canon_gather<double>(top.g, top.x64, top.bw64, nvn, npn, main);
    rc = cudaMemcpyAsync(x_host, top.bw64, size_t(3 * nvn + npn) * 8, cudaMemcpyDeviceToHost, main) == cudaSuccess
             ? HHG_OK : fail(HHG_ECUDA, "solution copy");
  }
  if (rc == HHG_OK && stats) rc = fill_stats(pb, prm, kernels, stats);
  cudaStreamSynchronize(pb->aux);
  cudaStreamSynchronize(pb->hp);
  if (rc != HHG_OK) {
    cudaStreamSynchronize(main);
    return rc;
  }
  HHG_CUDA(cudaStreamSynchronize(main));
  return HHG_OK;
}

// ================================================ learned coarse correction API
namespace {
int check_nn(const hhg_problem* pb) {
  if (!pb) return fail(HHG_EINVAL, "null problem");
  if (pb->nn_h <= 0) return fail(HHG_ESTATE, "problem created without nn_hidden");
  if (!pb->bound) return fail(HHG_ESTATE, "problem has no workspace bound");
  return HHG_OK;
}
}  // namespace

extern "C" int hhg_coarse_nn_size(const hhg_problem* pb, int* n, int64_t* n_params) {
  if (!pb || !n || !n_params) return fail(HHG_EINVAL, "null argument");
  if (pb->nn_h <= 0) return fail(HHG_ESTATE, "problem created without nn_hidden");
  *n = pb->nn_n;
  *n_params = pb->nn_P;
  return HHG_OK;
}

extern "C" int hhg_coarse_nn_set_params(hhg_problem* pb, const float* params) {
  HHG_TRY(check_nn(pb));
  if (!params) return fail(HHG_EINVAL, "null params");
  HHG_CUDA(cudaMemcpyAsync(pb->nn_params, params, size_t(pb->nn_P) * 4, cudaMemcpyHostToDevice, pb->stream));
  HHG_CUDA(cudaMemsetAsync(pb->nn_m, 0, size_t(pb->nn_P) * 4, pb->stream));
  HHG_CUDA(cudaMemsetAsync(pb->nn_v, 0, size_t(pb->nn_P) * 4, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  pb->nn_step = 0;
  return HHG_OK;
}

extern "C" int hhg_coarse_nn_get_params(hhg_problem* pb, float* params) {
  HHG_TRY(check_nn(pb));
  if (!params) return fail(HHG_EINVAL, "null params");
  HHG_CUDA(cudaMemcpyAsync(params, pb->nn_params, size_t(pb->nn_P) * 4, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  return HHG_OK;
}

extern "C" int hhg_coarse_nn_grad(hhg_problem* pb, const float* X, const float* T, int B, double* loss, float* grads) {
  HHG_TRY(check_nn(pb));
  if (!X || !T || !loss || !grads || B < 1 || B > pb->nn_B || B > pb->nn_S)
    return fail(HHG_EINVAL, "hhg_coarse_nn_grad: bad arguments (1 <= B <= nn_batch)");
  const int n = pb->nn_n;
  HHG_CUDA(cudaMemcpyAsync(pb->nn_X, X, size_t(B) * n * 4, cudaMemcpyHostToDevice, pb->stream));
  HHG_CUDA(cudaMemcpyAsync(pb->nn_T, T, size_t(B) * n * 4, cudaMemcpyHostToDevice, pb->stream));
  nn_forward(pb, pb->nn_X, B, pb->nn_H1, pb->nn_H2, pb->nn_Y);
  nn_backward(pb, pb->nn_X, pb->nn_T, B);
  const int nb = nn_mse(pb->nn_Y, pb->nn_T, int64_t(B) * n, 0.f, nullptr, pb->nn_part, pb->stream);
  HHG_CHECK_LAUNCH();
  std::vector<double> part(static_cast<size_t>(nb));
  HHG_CUDA(cudaMemcpyAsync(part.data(), pb->nn_part, part.size() * 8, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaMemcpyAsync(grads, pb->nn_grads, size_t(pb->nn_P) * 4, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  double sum = 0.0;
  for (double v : part) sum += v;
  *loss = sum / (double(B) * n);
  return HHG_OK;
}

extern "C" int hhg_coarse_nn_train(hhg_problem* pb, const hhg_nn_cfg* cfg, hhg_nn_report* rep) {
  HHG_TRY(check_nn(pb));
  if (!cfg || cfg->epochs < 1 || cfg->batch < 1 || cfg->batch > pb->nn_B || cfg->n_train < 1 ||
      cfg->n_train >= pb->nn_S || !(cfg->lr > 0) || cfg->smooth_frac < 0 || cfg->smooth_frac > 1)
    return fail(HHG_EINVAL, "hhg_coarse_nn_train: bad configuration (batch <= nn_batch, n_train < nn_samples)");
  const int n = pb->nn_n, S = pb->nn_S;
  cudaEvent_t e0, e1;
  HHG_CUDA(cudaEventCreate(&e0));
  HHG_CUDA(cudaEventCreate(&e1));
  HHG_CUDA(cudaEventRecord(e0, pb->stream));
  // random unit defects and the plain coarse solve of each: T = X Z^T
  const int nu = n - int((pb->lv[0].g.nx + 1) * int64_t(pb->lv[0].g.ny + 1) * (pb->lv[0].g.nz + 1));
  int R = 0;                                       // recorded defects kept in samples [0, R)
  if (cfg->recorded) {
    unsigned long long cnt = 0;
    HHG_CUDA(cudaMemcpyAsync(&cnt, pb->nn_counts + 2, 8, cudaMemcpyDeviceToHost, pb->stream));
    HHG_CUDA(cudaStreamSynchronize(pb->stream));
    R = int(std::min<unsigned long long>(cnt, unsigned(S)));
  }
  if (R < S)
    nn_samples(pb->nn_X + int64_t(R) * n, S - R, n, nu, pb->nn_mlp, pb->lv[0].ml_sum, cfg->seed, pb->nn_xyz,
               cfg->smooth_frac, pb->stream);
  nn_gemm(false, true, S, n, n, 1.f, pb->nn_X, n, pb->nn_Z, n, 0.f, pb->nn_T, n, pb->stream);
  {
    // scale the targets to unit RMS; inference multiplies by the inverse
    launch_reduce<float>(RED_SQ, pb->nn_T, nullptr, nullptr, int64_t(S) * n, pb->partials, pb->max_blocks,
                         pb->nn_scal + 4, pb->stream);
    double ms = 0.0;
    HHG_CUDA(cudaMemcpyAsync(&ms, pb->nn_scal + 4, 8, cudaMemcpyDeviceToHost, pb->stream));
    HHG_CUDA(cudaStreamSynchronize(pb->stream));
    ms /= double(S) * n;
    pb->nn_tscale = ms > 0 ? 1.0 / std::sqrt(ms) : 1.0;
    nn_scale(pb->nn_T, int64_t(S) * n, float(pb->nn_tscale), pb->stream);
  }
  double first_loss = 0.0, last_loss = 0.0, val_rel = 0.0;
  // mean squared error and mean relative error of the network on samples [first, first + count)
  auto eval = [&](int first, int count, double& mse, double& rel) -> int {
    double se = 0.0, rs = 0.0;
    for (int s0 = first; s0 < first + count; s0 += pb->nn_B) {
      const int bsz = std::min(pb->nn_B, first + count - s0);
      nn_forward(pb, pb->nn_X + int64_t(s0) * n, bsz, pb->nn_H1, pb->nn_H2, pb->nn_Y);
      std::vector<float> y(size_t(bsz) * n), t(size_t(bsz) * n);
      HHG_CUDA(cudaMemcpyAsync(y.data(), pb->nn_Y, y.size() * 4, cudaMemcpyDeviceToHost, pb->stream));
      HHG_CUDA(cudaMemcpyAsync(t.data(), pb->nn_T + int64_t(s0) * n, t.size() * 4, cudaMemcpyDeviceToHost, pb->stream));
      HHG_CUDA(cudaStreamSynchronize(pb->stream));
      for (int b = 0; b < bsz; ++b) {
        double num = 0.0, den = 0.0;
        for (int i = 0; i < n; ++i) {
          const double d = double(y[size_t(b) * n + i]) - t[size_t(b) * n + i];
          num += d * d;
          den += double(t[size_t(b) * n + i]) * t[size_t(b) * n + i];
        }
        se += num;
        rs += den > 0 ? std::sqrt(num / den) : 0.0;
      }
    }
    mse = se / (double(count) * n);
    rel = rs / count;
    return HHG_OK;
  };
  double dummy;
  HHG_TRY(eval(0, cfg->n_train, first_loss, dummy));
  for (int ep = 0; ep < cfg->epochs; ++ep)
    for (int s0 = 0; s0 < cfg->n_train; s0 += cfg->batch) {
      const int bsz = std::min(cfg->batch, cfg->n_train - s0);
      const float* X = pb->nn_X + int64_t(s0) * n;
      nn_forward(pb, X, bsz, pb->nn_H1, pb->nn_H2, pb->nn_Y);
      nn_backward(pb, X, pb->nn_T + int64_t(s0) * n, bsz);
      nn_adam(pb->nn_params, pb->nn_grads, pb->nn_m, pb->nn_v, pb->nn_P, float(cfg->lr), ++pb->nn_step, pb->stream);
    }
  HHG_CHECK_LAUNCH();
  HHG_CUDA(cudaEventRecord(e1, pb->stream));
  HHG_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HHG_TRY(eval(0, cfg->n_train, last_loss, dummy));
  double val_mse;
  HHG_TRY(eval(cfg->n_train, S - cfg->n_train, val_mse, val_rel));
  if (rep) {
    rep->n = n;
    rep->n_params = pb->nn_P;
    rep->loss_first = first_loss;
    rep->loss_last = last_loss;
    rep->val_rel_err = val_rel;
    rep->train_ms = ms;
  }
  if (!std::isfinite(last_loss)) return fail(HHG_EDIVERGED, "training diverged");
  return HHG_OK;
}

extern "C" int hhg_coarse_nn_record(hhg_problem* pb, int on, int64_t* recorded) {
  HHG_TRY(check_nn(pb));
  if (on && !pb->nn_recording) HHG_CUDA(cudaMemsetAsync(pb->nn_counts + 2, 0, 8, pb->stream));
  pb->nn_recording = on != 0;
  for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
  pb->graphs.clear();
  if (recorded) {
    unsigned long long cnt = 0;
    HHG_CUDA(cudaMemcpyAsync(&cnt, pb->nn_counts + 2, 8, cudaMemcpyDeviceToHost, pb->stream));
    HHG_CUDA(cudaStreamSynchronize(pb->stream));
    *recorded = int64_t(cnt);
  }
  return HHG_OK;
}

extern "C" int hhg_coarse_nn_enable(hhg_problem* pb, int mode, double theta) {
  HHG_TRY(check_nn(pb));
  if (mode < 0 || mode > 3 || !(theta > 0)) return fail(HHG_EINVAL, "mode in {0,1,2,3}, theta > 0");
  pb->nn_mode = mode;
  pb->nn_theta = theta;
  for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
  pb->graphs.clear();
  return HHG_OK;
}

extern "C" int hhg_coarse_nn_counts(hhg_problem* pb, int64_t* accepted, int64_t* rejected) {
  HHG_TRY(check_nn(pb));
  unsigned long long c[2];
  HHG_CUDA(cudaMemcpyAsync(c, pb->nn_counts, 16, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaMemsetAsync(pb->nn_counts, 0, 16, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  if (accepted) *accepted = int64_t(c[0]);
  if (rejected) *rejected = int64_t(c[1]);
  return HHG_OK;
}

// ================================================================ autotuner
namespace {
template <class T>
int tune_level(hhg_problem* pb, Level& lv, int reps, T* xa, T* xb) {
  cudaEvent_t e0, e1;
  HHG_CUDA(cudaEventCreate(&e0));
  HHG_CUDA(cudaEventCreate(&e1));
  auto time_it = [&](auto&& fn) {
    for (int r = 0; r < 2; ++r) fn();
    cudaEventRecord(e0, pb->stream);
    for (int r = 0; r < reps; ++r) fn();
    cudaEventRecord(e1, pb->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
  };
  const int disc = pb->desc.disc, varnu = pb->desc.nu_a != 0.0 ? 1 : 0;
  // row kernels: FULL residual, one site per thread or four runs of 32
  // sites per warp
  const int threads[3] = {64, 128, 256}, planes[5] = {1, 2, 4, 8, 16};
  float best = 1e30f;
  // the plain kernels are timed first; the streaming kernels compete after
  for (int o = 0; o < 3; ++o) lv.shape.st_threads[o] = lv.shape.st64_threads[o] = 0;
  Shape bestS = lv.shape;
  for (int v : {1, 4})
    for (int t : threads)
      for (int kp : planes) {
        if (v > 1 && (t == 64 || kp > 4)) continue;
        Shape sh = lv.shape;
        sh.row_threads = t;
        sh.row_kplanes = kp;
        sh.row_sites = v;
        const float ms = time_it([&] {
          fast_rows<T>(disc, varnu, OP_FULL, lv.g, lv.op[OP_FULL], ftab<T>(lv, OP_FULL), MODE_RES, xa, xa, xb, 1.0,
                       sh, pb->stream);
        });
        if (ms < best) { best = ms; bestS.row_threads = t; bestS.row_kplanes = kp; bestS.row_sites = v; }
      }
  if (std::is_same<T, double>::value) {
    bestS.row_sites64 = bestS.row_sites;
  } else {
    // the FP64 residual of the mixed solve's refinement: its own choice of
    // sites per thread (FP64 arithmetic, not the loads, bounds it)
    float best64 = 1e30f;
    for (int v : {1, 4}) {
      Shape sh = bestS;
      sh.row_sites64 = v;
      const float ms = time_it([&] {
        fast_rows<double>(disc, varnu, OP_FULL, lv.g, lv.op[OP_FULL], ftab<double>(lv, OP_FULL), MODE_RES, lv.tmp64,
                          lv.tmp64, lv.bw64, 1.0, sh, pb->stream);
      });
      if (ms < best64) { best64 = ms; bestS.row_sites64 = v; }
    }
  }
  // the smoother's B^T and (B, -C) residual rows: their own shapes (24 short
  // rows on one input array; one long row on all of them)
  for (int op : {OP_BT, OP_BC}) {
    float bo = 1e30f;
    int bt = 0, bk = 0, bs = 0;
    for (int v : {1, 4})
      for (int t : threads)
        for (int kp : {1, 2, 4}) {
          if (v > 1 && t == 64) continue;
          Shape sh = bestS;
          if (op == OP_BT) { sh.bt_threads = t; sh.bt_kplanes = kp; sh.bt_sites = v; }
          else { sh.bc_threads = t; sh.bc_kplanes = kp; sh.bc_sites = v; }
          const float ms = time_it([&] {
            fast_rows<T>(disc, varnu, op, lv.g, lv.op[op], ftab<T>(lv, op), MODE_RES, xa, xa, xb, 1.0, sh, pb->stream);
          });
          if (ms < bo) { bo = ms; bt = t; bk = kp; bs = v; }
        }
    if (op == OP_BT) { bestS.bt_threads = bt; bestS.bt_kplanes = bk; bestS.bt_sites = bs; }
    else { bestS.bc_threads = bt; bestS.bc_kplanes = bk; bestS.bc_sites = bs; }
  }
  // the streaming kernels (stream.cu) against the best plain shape, for the
  // FULL residual and the smoother's B^T and (B, -C) rows (threads per block),
  // in the V-cycle precision and, for the mixed solve, the FP64 residual
  {
    const int sops[3] = {OP_FULL, OP_BT, OP_BC};
    for (int o = 0; o < 3; ++o) {
      Shape sh = bestS;
      sh.st_threads[o] = 0;
      float bo = time_it([&] {
        fast_rows<T>(disc, varnu, sops[o], lv.g, lv.op[sops[o]], ftab<T>(lv, sops[o]), MODE_RES, xa, xa, xb, 1.0, sh,
                     pb->stream);
      });
      for (int v : {4, 2})
        for (int t : threads) {
          if (v == 2 && sizeof(T) == 8) continue;
          sh.st_threads[o] = t;
          sh.st_sites[o] = v;
          if (!stream_op<T>(pb, lv, sh, sops[o], MODE_RES, xa, xa, xb)) continue;
          const float ms = time_it([&] { stream_op<T>(pb, lv, sh, sops[o], MODE_RES, xa, xa, xb); });
          if (ms < bo) { bo = ms; bestS.st_threads[o] = t; bestS.st_sites[o] = v; }
        }
      if (std::is_same<T, double>::value) bestS.st64_threads[o] = bestS.st_threads[o];
    }
    if (!std::is_same<T, double>::value) {
      Shape sh = bestS;
      sh.st64_threads[0] = 0;
      float bo = time_it([&] {
        fast_rows<double>(disc, varnu, OP_FULL, lv.g, lv.op[OP_FULL], ftab<double>(lv, OP_FULL), MODE_RES, lv.tmp64,
                          lv.tmp64, lv.bw64, 1.0, sh, pb->stream);
      });
      for (int t : threads) {
        sh.st64_threads[0] = t;
        if (!stream_op<double>(pb, lv, sh, OP_FULL, MODE_RES, lv.tmp64, lv.tmp64, lv.bw64)) continue;
        const float ms = time_it([&] { stream_op<double>(pb, lv, sh, OP_FULL, MODE_RES, lv.tmp64, lv.tmp64, lv.bw64); });
        if (ms < bo) { bo = ms; bestS.st64_threads[0] = t; }
      }
    }
  }
  // Gauss-Seidel kernels: one forward sweep, 1, 2 or 4 lanes per site; the
  // lanes of the vertex colours and of the edge groups are then chosen apart
  best = 1e30f;
  auto sweep = [&](const Shape& sh, bool vertex, bool edges) {
    if (vertex)
      for (int c = 0; c < 4; ++c) fast_gs<T>(disc, varnu, lv.g, ftab<T>(lv, OP_A), 0, c, 1.0, xb, xa, sh, pb->stream);
    if (edges)
      for (int gg = 1; gg < lv.g.G; ++gg) fast_gs<T>(disc, varnu, lv.g, ftab<T>(lv, OP_A), gg, -1, 1.0, xb, xa, sh, pb->stream);
  };
  for (int nl : {1, 2, 4})
    for (int t : threads) {
      Shape sh = bestS;
      sh.gs_threads = t;
      sh.gs_lanes = sh.gs_lanes0 = nl;
      const float ms = time_it([&] { sweep(sh, true, true); });
      if (ms < best) { best = ms; bestS.gs_threads = t; bestS.gs_lanes = bestS.gs_lanes0 = nl; }
    }
  if (lv.g.G > 1) {
    float bv = 1e30f, be = 1e30f;
    int lv0 = bestS.gs_lanes0, tv0 = bestS.gs_threads, le = bestS.gs_lanes, te = bestS.gs_threads;
    for (int nl : {1, 2, 4})
      for (int t : threads) {
        Shape sh = bestS;
        sh.gs_lanes = sh.gs_lanes0 = nl;
        sh.gs_threads = t;
        sh.gs_threads0 = 0;
        const float mv = time_it([&] { sweep(sh, true, false); });
        const float me = time_it([&] { sweep(sh, false, true); });
        if (mv < bv) { bv = mv; lv0 = nl; tv0 = t; }
        if (me < be) { be = me; le = nl; te = t; }
      }
    bestS.gs_lanes0 = lv0;
    bestS.gs_threads0 = tv0;
    bestS.gs_lanes = le;
    bestS.gs_threads = te;
  }
  // launch order of a smoothing step's phases: every phase on all three
  // components, or component by component (two forward sweeps each)
  {
    auto sweeps = [&](const Shape& sh) {
      for (int c = sh.gs_comp_major ? 0 : -1; c < (sh.gs_comp_major ? 3 : 0); ++c)
        for (int r = 0; r < 2; ++r) {
          for (int cc = 0; cc < 4; ++cc)
            fast_gs<T>(disc, varnu, lv.g, ftab<T>(lv, OP_A), 0, cc, 1.0, xb, xa, sh, pb->stream, c);
          for (int gg = 1; gg < lv.g.G; ++gg)
            fast_gs<T>(disc, varnu, lv.g, ftab<T>(lv, OP_A), gg, -1, 1.0, xb, xa, sh, pb->stream, c);
        }
    };
    Shape sh = bestS;
    sh.gs_comp_major = 0;
    const float m0 = time_it([&] { sweeps(sh); });
    sh.gs_comp_major = 1;
    const float m1 = time_it([&] { sweeps(sh); });
    bestS.gs_comp_major = m1 < m0 ? 1 : 0;
  }
  lv.shape = bestS;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HHG_CUDA(cudaMemsetAsync(xa, 0, size_t(lv.nvec()) * sizeof(T), pb->stream));
  HHG_CUDA(cudaMemsetAsync(xb, 0, size_t(lv.nvec()) * sizeof(T), pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  return HHG_OK;
}
// the smoother of a level: per-phase kernels against the resident smoother
// on every CTA count that holds the level (two Uzawa iterations, xi = 2)
template <class T>
int tune_smoother(hhg_problem* pb, Level& lv, int reps, T* x, const T* b, T* tmp) {
  const int prec = prec_index<T>();
  const size_t bytes = size_t(lv.nvec()) * sizeof(T);
  hhg_params prm{1, 1, 0, 1, HHG_AHAT_F, 2, 0.5};
  cudaEvent_t e0, e1;
  HHG_CUDA(cudaEventCreate(&e0));
  HHG_CUDA(cudaEventCreate(&e1));
  int best_c = 0, best_t = kResidentThreads;
  float best = 1e30f;
  for (int cand = 0; cand < 16; ++cand) {
    const int C = cand == 0 ? 0 : 1 << ((cand - 1) / 3), th = cand == 0 ? kResidentThreads : 256 << ((cand - 1) % 3);
    if (C > kResidentMaxCtas || (C > 0 && !resident_feasible(prec, lv.g, C))) continue;
    HHG_TRY(set_resident(pb, lv, prec, C, th));
    HHG_CUDA(cudaMemsetAsync(x, 0, bytes, pb->stream));
    HHG_CUDA(cudaMemsetAsync(tmp, 0, bytes, pb->stream));
    HHG_TRY(uzawa<T>(pb, lv, prm, 2, x, b, tmp));
    cudaEventRecord(e0, pb->stream);
    for (int r = 0; r < reps; ++r) HHG_TRY(uzawa<T>(pb, lv, prm, 2, x, b, tmp));
    cudaEventRecord(e1, pb->stream);
    HHG_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_c = C; best_t = th; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  HHG_TRY(set_resident(pb, lv, prec, best_c, best_t));
  HHG_CUDA(cudaMemsetAsync(x, 0, bytes, pb->stream));
  HHG_CUDA(cudaMemsetAsync(tmp, 0, bytes, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  return HHG_OK;
}
}  // namespace

extern "C" int hhg_autotune(hhg_problem* pb, int reps, int* shapes_out) {
  HHG_TRY(check_level(pb, pb ? pb->desc.L : 0));
  if (reps < 1) return fail(HHG_EINVAL, "reps must be positive");
  const bool mixed = pb->desc.solve == HHG_SOLVE_MIXED;
  const double wu = pb->wu_counted;
  for (int l = pb->desc.coarse_level; l <= pb->desc.L; ++l) {
    Level& lv = pb->L(l);
    if (mixed) {
      HHG_TRY(tune_level<float>(pb, lv, reps, lv.tmp32, lv.b32));
      HHG_TRY(tune_smoother<float>(pb, lv, reps, lv.x32, lv.b32, lv.tmp32));
    } else {
      HHG_TRY(tune_level<double>(pb, lv, reps, lv.tmp64, lv.bw64));
      HHG_TRY(tune_smoother<double>(pb, lv, reps, lv.bw64, lv.rhs, lv.tmp64));
    }
    if (shapes_out) {
      int* o = shapes_out + 16 * (l - pb->desc.coarse_level);
      o[0] = lv.shape.row_threads; o[1] = lv.shape.row_kplanes; o[2] = lv.shape.gs_threads;
      o[3] = lv.rctas[mixed ? HHG_FP32 : HHG_FP64];
      o[4] = lv.rthreads[mixed ? HHG_FP32 : HHG_FP64];
      o[5] = lv.shape.st_threads[0];
      o[6] = lv.shape.row_sites;
      o[7] = lv.shape.gs_lanes;
      o[8] = lv.shape.gs_lanes0;
      o[9] = lv.shape.bt_threads; o[10] = lv.shape.bt_kplanes; o[11] = lv.shape.bt_sites;
      o[12] = lv.shape.bc_threads; o[13] = lv.shape.bc_kplanes; o[14] = lv.shape.bc_sites;
      o[15] = lv.shape.gs_threads0 ? lv.shape.gs_threads0 : lv.shape.gs_threads;
    }
  }
  pb->wu_counted = wu;
  for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
  pb->graphs.clear();
  return HHG_OK;
}

// ================================================================== batches
struct hhg_batch {
  std::vector<hhg_problem*> pbs;
  std::vector<cudaStream_t> streams;      // one capture stream per problem
  std::vector<cudaEvent_t> events;        // join events
  cudaEvent_t fork = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<hhg_params> key;            // parameters the graph was recorded with
  int64_t kernels = 0;
  int64_t ops = 0;                        // kernels of the problems' own sequences
  int grouping = -1;                      // hhg_batch_set_grouping (-1: automatic)
  int used_grouping = -1;                 // the grouping of the current graph
  std::vector<std::unique_ptr<Recorder>> recs;   // per cohort: device tables and work items of the merged launches
  ~hhg_batch() {
    if (exec) cudaGraphExecDestroy(exec);
    for (auto e : events) cudaEventDestroy(e);
    for (auto s : streams) cudaStreamDestroy(s);
    if (fork) cudaEventDestroy(fork);
  }
};

extern "C" int hhg_batch_create(hhg_problem* const* problems, int n, hhg_batch** out) {
  if (!problems || n < 1 || !out) return fail(HHG_EINVAL, "hhg_batch_create: bad arguments");
  auto bt = std::make_unique<hhg_batch>();
  for (int i = 0; i < n; ++i) {
    hhg_problem* pb = problems[i];
    if (!pb || !pb->bound) return fail(HHG_ESTATE, "hhg_batch_create: every problem must be bound");
    for (int l = pb->desc.coarse_level; l <= pb->desc.L; ++l)
      if (!pb->L(l).has_rhs) return fail(HHG_ESTATE, "hhg_batch_create: hhg_set_rhs missing on a level");
    for (hhg_problem* q : bt->pbs)
      if (q == pb) return fail(HHG_EINVAL, "hhg_batch_create: a problem appears twice");
    bt->pbs.push_back(pb);
    cudaStream_t s;
    HHG_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    bt->streams.push_back(s);
    cudaEvent_t e;
    HHG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    bt->events.push_back(e);
  }
  HHG_CUDA(cudaEventCreateWithFlags(&bt->fork, cudaEventDisableTiming));
  // one launch shape per (discretisation, level) across the batch, so that the
  // problems' kernels can share launches: that of the problem with the most
  // DoFs on the level; the resident smoother keeps each problem's CTA count
  // (it depends on the level's size) and takes, per CTA count, the largest
  // problem's CTA size
  for (hhg_problem* pb : bt->pbs) {
    for (int l = pb->desc.coarse_level; l <= pb->desc.L; ++l) {
      const hhg_problem* big = pb;
      for (const hhg_problem* q : bt->pbs)
        if (q->desc.disc == pb->desc.disc && l >= q->desc.coarse_level && l <= q->desc.L &&
            const_cast<hhg_problem*>(q)->L(l).n_dofs() > const_cast<hhg_problem*>(big)->L(l).n_dofs())
          big = q;
      Level& lv = pb->L(l);
      lv.shape = const_cast<hhg_problem*>(big)->L(l).shape;
      for (int pr = 0; pr < 2; ++pr) {
        const hhg_problem* bc = pb;
        for (const hhg_problem* q : bt->pbs)
          if (q->desc.disc == pb->desc.disc && l >= q->desc.coarse_level && l <= q->desc.L &&
              const_cast<hhg_problem*>(q)->L(l).rctas[pr] == lv.rctas[pr] &&
              const_cast<hhg_problem*>(q)->L(l).n_dofs() > const_cast<hhg_problem*>(bc)->L(l).n_dofs())
            bc = q;
        lv.rthreads[pr] = const_cast<hhg_problem*>(bc)->L(l).rthreads[pr];
      }
    }
    for (auto& kv : pb->graphs) cudaGraphExecDestroy(kv.second.exec);
    pb->graphs.clear();
  }
  *out = bt.release();
  return HHG_OK;
}

extern "C" int hhg_batch_destroy(hhg_batch* bt) {
  delete bt;
  return HHG_OK;
}

namespace {
bool same_params(const std::vector<hhg_params>& a, const hhg_params* b) {
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].nu_pre != b[i].nu_pre || a[i].nu_post != b[i].nu_post || a[i].nu_inc != b[i].nu_inc ||
        a[i].kappa != b[i].kappa || a[i].ahat != b[i].ahat || a[i].xi != b[i].xi || a[i].omega_inv != b[i].omega_inv)
      return false;
  return true;
}
}  // namespace

namespace {
// every problem's FMG on its own branch of one graph (batches whose problems
// use the learned coarse correction, whose kernels are not recorded)
int capture_branches(hhg_batch* bt, const hhg_params* params, cudaGraph_t* graph) {
  const int n = int(bt->pbs.size());
  cudaStream_t cap = bt->streams[0];
  const int64_t l0 = g_launches;
  HHG_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  int rc = HHG_OK;
  cudaError_t ce = cudaEventRecord(bt->fork, cap);
  for (int i = 0; i < n && rc == HHG_OK && ce == cudaSuccess; ++i) {
    hhg_problem* pb = bt->pbs[i];
    if (i > 0) ce = cudaStreamWaitEvent(bt->streams[i], bt->fork, 0);
    if (ce != cudaSuccess) break;
    cudaStream_t keep = pb->stream;
    pb->stream = bt->streams[i];
    rc = fmg_core(pb, &params[i]);
    pb->stream = keep;
    if (i > 0 && rc == HHG_OK) {
      ce = cudaEventRecord(bt->events[i], bt->streams[i]);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, bt->events[i], 0);
    }
  }
  cudaError_t ee = cudaStreamEndCapture(cap, graph);
  if (rc != HHG_OK) return rc;
  if (ce != cudaSuccess || ee != cudaSuccess)
    return fail(HHG_ECUDA, std::string("batch capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee));
  bt->kernels = bt->ops = g_launches - l0;
  return HHG_OK;
}

struct RecordScope {
  explicit RecordScope(Recorder* r) { g_rec = r; }
  ~RecordScope() { g_rec = nullptr; }
};

// record every problem's FMG, merge the sequences into shared launches over
// all problems (batch.h) and capture those launches.  The problems form
// cohorts; each cohort's merged launches are one chain on its own branch of
// the graph, and the cohorts run side by side.  Grouping 0: a cohort is the
// problems whose kernel sequences are the same op for op (discretisation,
// precision, coarse and finest level, viscosity model, smoothing tuple, and
// which levels smooth in one resident launch with how many CTAs).  Grouping
// 1: the problems with the same discretisation, precision, coarse level,
// viscosity model and smoothing tuple, whatever their size (fewer, longer
// chains; the merge aligns their sequences as far as they agree)
// cohort of every problem under grouping 0 or 1; returns the cohort count
int cohorts_of(const hhg_batch* bt, const hhg_params* params, int grouping, std::vector<int>& cohort) {
  const int n = int(bt->pbs.size());
  std::vector<std::vector<int>> keys;
  cohort.assign(n, 0);
  for (int i = 0; i < n; ++i) {
    hhg_problem* pb = bt->pbs[i];
    const hhg_params& p = params[i];
    const int prec = pb->desc.solve == HHG_SOLVE_FP64 ? HHG_FP64 : HHG_FP32;
    std::vector<int> key = {pb->desc.disc, pb->desc.solve, pb->desc.coarse_level, pb->desc.nu_a != 0.0 ? 1 : 0,
                            p.nu_pre, p.nu_post, p.nu_inc, p.kappa, p.ahat, p.xi};
    if (grouping == 0) {
      key.push_back(pb->desc.L);
      for (int l = pb->desc.coarse_level; l <= pb->desc.L; ++l) key.push_back(pb->L(l).rctas[prec]);
    }
    auto it = std::find(keys.begin(), keys.end(), key);
    cohort[i] = int(it - keys.begin());
    if (it == keys.end()) keys.push_back(key);
  }
  return int(keys.size());
}

int capture_merged(hhg_batch* bt, const hhg_params* params, int grouping, cudaGraph_t* graph) {
  const int n = int(bt->pbs.size());
  std::vector<int> cohort;
  const int nc = cohorts_of(bt, params, grouping, cohort);
  std::vector<std::unique_ptr<Recorder>> recs(nc);
  std::vector<std::vector<BatchLaunch>> launches(nc);
  int64_t batched = 0;
  for (int c = 0; c < nc; ++c) {
    recs[c] = std::make_unique<Recorder>();
    {
      RecordScope scope(recs[c].get());
      int slot = 0;
      for (int i = 0; i < n; ++i) {
        if (cohort[i] != c) continue;
        recs[c]->begin(slot++);
        HHG_TRY(fmg_core(bt->pbs[i], &params[i]));
      }
    }
    const int me = recs[c]->merge(launches[c]);
    if (me != 0) return fail(HHG_ECUDA, std::string("batch merge: ") + cudaGetErrorString(cudaError_t(me)));
    batched += recs[c]->batched_kernels();
  }
  // function attributes before the capture: per kernel the largest dynamic
  // shared memory of its launches, and non-portable cluster sizes
  std::map<const void*, size_t> smem_of;
  std::set<const void*> big_cluster;
  for (const auto& ls : launches)
    for (const BatchLaunch& l : ls) {
      if (l.native) continue;
      smem_of[l.fn] = std::max(smem_of[l.fn], l.smem);
      if (l.cluster > 8) big_cluster.insert(l.fn);
    }
  for (const auto& kv : smem_of)
    if (kv.second > 48 * 1024)
      HHG_CUDA(cudaFuncSetAttribute(kv.first, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kv.second)));
  for (const void* fn : big_cluster) HHG_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaStream_t cap = bt->streams[0];
  int64_t merged = 0;
  const int64_t l0 = g_launches;
  HHG_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
  cudaError_t ce = cudaEventRecord(bt->fork, cap);
  for (int c = 0; c < nc && ce == cudaSuccess; ++c) {
    cudaStream_t sc = bt->streams[c];
    if (c > 0) ce = cudaStreamWaitEvent(sc, bt->fork, 0);
    for (size_t q = 0; q < launches[c].size() && ce == cudaSuccess; ++q) {
      ce = launch_merged(launches[c][q], recs[c]->items(), sc);
      if (!launches[c][q].native) ++merged;
    }
    if (c > 0 && ce == cudaSuccess) {
      ce = cudaEventRecord(bt->events[c], sc);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, bt->events[c], 0);
    }
  }
  cudaError_t ee = cudaStreamEndCapture(cap, graph);
  if (ce != cudaSuccess || ee != cudaSuccess)
    return fail(HHG_ECUDA, std::string("batch capture: ") + cudaGetErrorString(ce != cudaSuccess ? ce : ee));
  bt->kernels = merged + (g_launches - l0);
  bt->ops = batched + (g_launches - l0);
  bt->recs = std::move(recs);
  return HHG_OK;
}
}  // namespace

extern "C" int hhg_batch_fmg_solve(hhg_batch* bt, const hhg_params* params, void* stream, int64_t* kernels) {
  if (!bt || !params) return fail(HHG_EINVAL, "hhg_batch_fmg_solve: null argument");
  const int n = int(bt->pbs.size());
  for (int i = 0; i < n; ++i) HHG_TRY(check_params(&params[i]));
  cudaStream_t s0 = static_cast<cudaStream_t>(stream);
  if (!bt->exec || !same_params(bt->key, params)) {
    if (bt->exec) { cudaGraphExecDestroy(bt->exec); bt->exec = nullptr; }
    // automatic grouping: merge the cohorts of identical sequences when they
    // hold four problems each on average, else one branch per problem
    int grouping = bt->grouping;
    if (grouping < 0) {
      std::vector<int> cohort;
      grouping = n >= 4 * cohorts_of(bt, params, 0, cohort) ? 0 : 2;
    }
    bool plain = grouping != 2;
    for (hhg_problem* pb : bt->pbs) plain = plain && pb->nn_mode == 0 && !pb->nn_recording;
    cudaGraph_t graph = nullptr;
    const int rc = plain ? capture_merged(bt, params, grouping, &graph) : capture_branches(bt, params, &graph);
    bt->used_grouping = plain ? grouping : 2;
    if (rc != HHG_OK) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    cudaError_t ei = cudaGraphInstantiate(&bt->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return fail(HHG_ECUDA, std::string("batch graph instantiate: ") + cudaGetErrorString(ei));
    bt->key.assign(params, params + n);
  }
  HHG_CUDA(cudaGraphLaunch(bt->exec, s0));
  if (kernels) *kernels = bt->kernels;
  return HHG_OK;
}

extern "C" int hhg_batch_set_grouping(hhg_batch* bt, int grouping) {
  if (!bt || grouping < -1 || grouping > 2) return fail(HHG_EINVAL, "hhg_batch_set_grouping: bad arguments");
  if (grouping != bt->grouping && bt->exec) {
    cudaGraphExecDestroy(bt->exec);
    bt->exec = nullptr;
  }
  bt->grouping = grouping;
  return HHG_OK;
}

extern "C" int hhg_batch_launch_counts(const hhg_batch* bt, int64_t* launches, int64_t* problem_kernels) {
  if (!bt || !launches || !problem_kernels) return fail(HHG_EINVAL, "hhg_batch_launch_counts: null argument");
  *launches = bt->kernels;
  *problem_kernels = bt->ops;
  return HHG_OK;
}

extern "C" int hhg_batch_get_grouping(const hhg_batch* bt, int* grouping) {
  if (!bt || !grouping) return fail(HHG_EINVAL, "hhg_batch_get_grouping: null argument");
  *grouping = bt->used_grouping;
  return HHG_OK;
}

extern "C" int hhg_estimate_omega(hhg_problem* pb, int level, int iters, const double* v0, double* omega_inv) {
  HHG_TRY(check_level(pb, level));
  if (!v0 || !omega_inv || iters < 1) return fail(HHG_EINVAL, "bad arguments");
  Level& lv = pb->L(level);
  const Geo& g = lv.g;
  const int64_t po = p_offset(lv);
  std::vector<double> h(size_t(lv.nvec()), 0.0);
  for_each_pressure_node(g, [&](int64_t ci, int64_t site) { h[size_t(po + site)] = v0[ci]; });
  double* V1 = lv.tmp64;   // (z_u | v_p)
  double* V2 = lv.x64;     // (y_u | -v_p)
  double* Wv = lv.bw64;    // (. | w_p)
  HHG_CUDA(cudaMemcpyAsync(V1, h.data(), h.size() * 8, cudaMemcpyHostToDevice, pb->stream));
  HHG_TRY(project_pressure(pb, lv, V1));
  double nr[2];
  HHG_TRY(norms_of(pb, lv, HHG_FP64, V1, nr));
  launch_xpby<double>(V1 + po, 1.0 / nr[1] - 1.0, V1 + po, V1 + po, g.arr, pb->stream);
  std::vector<std::pair<int, int>> phases;
  for (int c = 0; c < 4; ++c) phases.push_back({0, c});
  for (int gg = 1; gg < g.G; ++gg) phases.push_back({gg, -1});
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    HHG_TRY(apply_op<double>(pb, lv, OP_BT, MODE_SET, V1, nullptr, V1));          // z = B^T v
    HHG_CUDA(cudaMemsetAsync(V2, 0, size_t(lv.nvec()) * 8, pb->stream));
    for (auto& ph : phases) launch_gs<double>(g, lv.op[OP_A], ph.first, ph.second, lv.inv_diag[ph.first], V2, V1, pb->stream);
    for (auto r = phases.rbegin(); r != phases.rend(); ++r)
      launch_gs<double>(g, lv.op[OP_A], r->first, r->second, lv.inv_diag[r->first], V2, V1, pb->stream);
    launch_axpy<double>(-1.0, V1 + po, V2 + po, g.arr, pb->stream);                // V2_p = -v
    HHG_TRY(apply_op<double>(pb, lv, OP_BC, MODE_SET, V2, nullptr, Wv));           // w = B y + C v
    launch_xpby<double>(Wv + po, 0.0, Wv + po, Wv + po, g.arr, pb->stream);
    // w <- M_L(1/nu)^{-1} w : multiply by inv_mlhat through the pressure update
    // kernel applied to a zero vector: 0 - (w * inv_ml) * (-1)
    HHG_CUDA(cudaMemsetAsync(V1 + po, 0, size_t(g.arr) * 8, pb->stream));
    launch_pupdate<double>(g, V1 + po, Wv + po, lv.inv_mlhat, -1.0, pb->stream);
    HHG_CHECK_LAUNCH();
    HHG_TRY(norms_of(pb, lv, HHG_FP64, V1, nr));
    lam = nr[1];
    if (!(lam > 0) || !std::isfinite(lam)) return fail(HHG_EDIVERGED, "power iteration broke down");
    launch_xpby<double>(V1 + po, 1.0 / lam - 1.0, V1 + po, V1 + po, g.arr, pb->stream);
  }
  HHG_CUDA(cudaMemsetAsync(lv.tmp64, 0, size_t(lv.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaMemsetAsync(lv.x64, 0, size_t(lv.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaMemsetAsync(lv.bw64, 0, size_t(lv.nvec()) * 8, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  *omega_inv = lam;
  return HHG_OK;
}

extern "C" int hhg_error_norms(hhg_problem* pb, int level, const void* x, const double* u_exact, const double* p_exact,
                               double* err_u, double* err_p) {
  HHG_TRY(check_level(pb, level));
  if (!pb->desc.error_level || level != pb->desc.L) return fail(HHG_EINVAL, "error norms need error_level and level == L");
  if (!x || !u_exact || !p_exact || !err_u || !err_p) return fail(HHG_EINVAL, "null argument");
  Level& c = pb->L(level);
  Level& f = pb->L(level + 1);
  const Geo& g = f.g;
  launch_xpby<double>(static_cast<const double*>(x), 1.0, c.W, c.tmp64, c.nvec(), pb->stream);
  HHG_CUDA(cudaMemsetAsync(f.x64, 0, size_t(f.nvec()) * 8, pb->stream));
  HHG_TRY(prolong_add<double>(pb, level + 1, c.tmp64, f.x64, false));
  // exact nodal values on level l+1
  const int64_t nvn = velocity_nodes(g), npn = pressure_nodes(g);
  HHG_CUDA(cudaMemcpyAsync(f.bw64, u_exact, size_t(3 * nvn) * 8, cudaMemcpyHostToDevice, pb->stream));
  HHG_CUDA(cudaMemcpyAsync(f.bw64 + 3 * nvn, p_exact, size_t(npn) * 8, cudaMemcpyHostToDevice, pb->stream));
  HHG_CUDA(cudaMemsetAsync(f.tmp64, 0, size_t(f.nvec()) * 8, pb->stream));
  launch_canon_scatter<double>(g, f.bw64, f.tmp64, nvn, npn, true, false, pb->stream);
  launch_xpby<double>(f.tmp64, -1.0, f.x64, f.tmp64, f.nvec(), pb->stream);        // d = x* - I x
  HHG_TRY(project_pressure(pb, f, f.tmp64));
  HHG_TRY(apply_op<double>(pb, f, OP_MASS, MODE_SET, f.tmp64, nullptr, f.x64));    // M d
  const int64_t po = p_offset(f);
  launch_reduce<double>(RED_DOT, f.tmp64, f.x64, nullptr, po, pb->partials, pb->max_blocks, pb->scal + 3, pb->stream);
  launch_reduce<double>(RED_DOT, f.tmp64 + po, f.x64 + po, nullptr, g.arr, pb->partials, pb->max_blocks, pb->scal + 4, pb->stream);
  HHG_CHECK_LAUNCH();
  double e2[2];
  HHG_CUDA(cudaMemcpyAsync(e2, pb->scal + 3, 16, cudaMemcpyDeviceToHost, pb->stream));
  HHG_CUDA(cudaStreamSynchronize(pb->stream));
  *err_u = std::sqrt(std::max(e2[0], 0.0));
  *err_p = std::sqrt(std::max(e2[1], 0.0));
  HHG_CUDA(cudaMemsetAsync(c.tmp64, 0, size_t(c.nvec()) * 8, pb->stream));
  return HHG_OK;
}
