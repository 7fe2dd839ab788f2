"""GPU parity at the benchmarked problem sizes, through the C ABI.

The oracle cannot assemble level-6/7 operators, so single rows of
Eq. stokes-discrete are computed from their definition (oracle/sampled.py:
the element contributions of the micro tetrahedra around the row's DoF) and
compared entrywise with the library's apply and residual on the same seeded
input.  The problems are those the benchmark runs, set up and autotuned the
same way (the launch shapes under test are the autotuned ones):

  * P2-P1 Taylor-Hood on the 6-tetrahedron cube, levels 6 and 7;
  * P1-P1 PSPG on the 48-tetrahedron cube (2 x 2 x 2 Kuhn box) on level 7
    with nu = exp(a z), a drawn from seed 0.

About 2,000 rows per case cover every row kind (3 velocity components x
the DoF groups, and the pressure rows), the pressure rows on every face,
edge and corner of the box (their C terms are clipped to the domain), the
Dirichlet velocity rows (which must be 0), and the last planes, rows and
columns of the box.

Tolerances, entrywise, with s_i = sum_j |a_ij x_j| (returned by the oracle):
  * FP64: |y_i - y_i^oracle| <= 64 eps_64 s_i.  Rounding of a sum of at most
    ~160 products is bounded by (n eps) s_i; a wrong, missing or transposed
    term moves y_i by |a_ij x_j| ~ s_i / n, far above the bound.  The
    relative-norm form of the tolerance would be blind at smooth inputs
    (row sums of A and C vanish), so it is not used.
  * FP32 (the V-cycle precision): the kernel reads x rounded to FP32 (the
    oracle evaluates the same rounded x) with FP32 weights (relative error
    <= eps_32 / 2 each) and sums n <= 160 terms in FP32:
    |y_i - y_i^oracle| <= (n + 2) eps_32 s_i <= 256 eps_32 s_i.
"""
import numpy as np
import pytest
import torch

from gpu_helpers import rel

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps
EPS32 = float(np.finfo(np.float32).eps)
GROUP_OFF = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


def _viscosity_exponent():
    from hhg_inputs import draw_viscosity_exponent
    return draw_viscosity_exponent(0)


# (disc, box, H, L, coarse level, nu_a): the benchmark's problems
CASES = [
    ("P2P1", (1, 1, 1), 1.0, 6, 2, 0.0),
    ("P2P1", (1, 1, 1), 1.0, 7, 2, 0.0),
    ("P1P1", (2, 2, 2), 0.5, 7, 0, "seed0"),
]


def _pick_rows(dims, disc, rng, per_kind):
    """(field, canonical node) rows: random sites of every row kind plus the
    box's boundary classes and last planes."""
    nx, ny, nz = dims
    rows = []

    def extremes(n):
        return [0, 1, n - 1, n]

    if disc == "P2P1":
        a, b = 2 * nx + 1, 2 * ny + 1
        for c in range(3):
            for ox, oy, oz in GROUP_OFF:
                mi, mj, mk = nx - ox, ny - oy, nz - oz           # coarse index range of the group
                pts = [tuple(rng.integers(0, m + 1) for m in (mi, mj, mk)) for _ in range(per_kind)]
                pts += [(rng.integers(0, mi + 1), rng.integers(0, mj + 1), kk) for kk in (mk, max(mk - 1, 0))]
                pts += [(ii, jj, rng.integers(0, mk + 1)) for ii in (0, mi) for jj in (0, mj)]
                pts += [(mi, mj, mk), (max(mi - 1, 0), max(mj - 1, 0), max(mk - 1, 0))]
                for i, j, k in pts:
                    I, J, K = 2 * int(i) + ox, 2 * int(j) + oy, 2 * int(k) + oz
                    rows.append((c, I + a * (J + b * K)))
    else:
        a, b = nx + 1, ny + 1
        for c in range(3):
            pts = [tuple(rng.integers(0, m + 1) for m in (nx, ny, nz)) for _ in range(per_kind)]
            pts += [(rng.integers(0, nx + 1), rng.integers(0, ny + 1), kk) for kk in extremes(nz)]
            pts += [(ii, jj, rng.integers(0, nz + 1)) for ii in extremes(nx) for jj in (0, ny)]
            for i, j, k in pts:
                rows.append((c, int(i) + a * (int(j) + b * int(k))))
    # pressure rows: random, every face / edge / corner class, last planes
    a, b = nx + 1, ny + 1
    pts = [tuple(rng.integers(0, m + 1) for m in (nx, ny, nz)) for _ in range(per_kind * 2)]
    for ci in (0, 1, 2):
        for cj in (0, 1, 2):
            for ck in (0, 1, 2):
                pick = lambda cls, n: (0 if cls == 0 else n if cls == 2 else int(rng.integers(1, n)))
                for _ in range(4):
                    pts.append((pick(ci, nx), pick(cj, ny), pick(ck, nz)))
    pts += [(rng.integers(0, nx + 1), rng.integers(0, ny + 1), kk) for kk in extremes(nz)]
    for i, j, k in pts:
        rows.append((3, int(i) + a * (int(j) + b * int(k))))
    return rows


def _dirichlet_mask(info, disc):
    """Boundary flags of the canonical velocity nodes (index arithmetic)."""
    if disc == "P2P1":
        a, b, c = 2 * info.nx + 1, 2 * info.ny + 1, 2 * info.nz + 1
    else:
        a, b, c = info.nx + 1, info.ny + 1, info.nz + 1
    idx = np.arange(a * b * c, dtype=np.int64)
    I, J, K = idx % a, (idx // a) % b, idx // (a * b)
    return (I == 0) | (I == a - 1) | (J == 0) | (J == b - 1) | (K == 0) | (K == c - 1)


def _smooth_field(info, disc):
    """x = sin(pi X) sin(pi Y) sin(pi Z) (1 + c/2) on velocity component c
    (0 on the boundary) and cos(pi X) cos(pi Y) cos(pi Z) on the pressure
    nodes, canonical order, for a box mapped to the unit cube."""
    def coords(a, b, c):
        idx = np.arange(a * b * c, dtype=np.int64)
        return (idx % a) / (a - 1), ((idx // a) % b) / (b - 1), (idx // (a * b)) / (c - 1)
    if disc == "P2P1":
        X, Y, Z = coords(2 * info.nx + 1, 2 * info.ny + 1, 2 * info.nz + 1)
    else:
        X, Y, Z = coords(info.nx + 1, info.ny + 1, info.nz + 1)
    xp, yp, zp = coords(info.nx + 1, info.ny + 1, info.nz + 1)
    su = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    return np.concatenate([su * (1.0 + 0.5 * c) for c in range(3)] +
                          [np.cos(np.pi * xp) * np.cos(np.pi * yp) * np.cos(np.pi * zp)])


def _gather(vec, rows, nv):
    return np.array([vec[f * nv + n] if f < 3 else vec[3 * nv + n] for f, n in rows])


@pytest.mark.parametrize("disc,box,H,L,lc,nu_a", CASES, ids=["P2P1-L6", "P2P1-L7", "P1P1-48tet-L7-visc"])
def test_fullsize_rows_match_oracle(disc, box, H, L, lc, nu_a):
    from oracle.sampled import sample_rows
    from paper_2010_13513_gb300 import hhg
    if nu_a == "seed0":
        nu_a = _viscosity_exponent()
    torch.cuda.set_stream(torch.cuda.Stream())
    pb = hhg.Problem(hhg.Mesh.box(*box, H), disc=disc, L=L, coarse_level=lc, solve="mixed", nu_a=nu_a)
    shapes = pb.autotune(reps=2)
    info = pb.layout(L)
    nv, npp = info.n_velocity_nodes, info.n_pressure_nodes
    rng = np.random.default_rng(11)
    vmask = np.tile(~_dirichlet_mask(info, disc), 3)
    x = rng.uniform(-1.0, 1.0, 3 * nv + npp)
    x[:3 * nv] *= vmask
    b = rng.uniform(-1.0, 1.0, 3 * nv + npp)
    b[:3 * nv] *= vmask
    rows = _pick_rows((info.nx, info.ny, info.nz), disc, rng, per_kind=70 if disc == "P2P1" else 500)
    assert len(rows) >= 2000
    ref, s = sample_rows(box, H, L, disc, x, rows, nu_a, with_abs=True)
    brow = _gather(b, rows, nv)
    dirichlet = s == 0.0
    assert dirichlet.any() and (~dirichlet).sum() > 1800

    # FP64 apply (the outer residual's precision)
    xd = pb.to_device(L, x)
    y = pb.new_vector(L)
    pb.apply(L, "FULL", xd, y)
    got = _gather(pb.to_host(L, y), rows, nv)
    err = np.abs(got - ref)
    assert np.all(err <= 64 * EPS64 * s), (float((err / np.maximum(s, 1e-300)).max()), shapes[L])
    assert np.all(got[dirichlet] == 0.0)

    # FP64 residual r = b - calA x and its norms
    r = pb.new_vector(L)
    nr = pb.residual(L, xd, pb.to_device(L, b), r, norms=True)
    rh = pb.to_host(L, r)
    gr = _gather(rh, rows, nv)
    assert np.all(np.abs(gr - (brow - ref)) <= 64 * EPS64 * (s + np.abs(brow)))
    assert nr[0] == pytest.approx(np.linalg.norm(rh[:3 * nv]), rel=1e-12)
    assert nr[1] == pytest.approx(np.linalg.norm(rh[3 * nv:]), rel=1e-12)
    del xd, y, r, rh

    # the mixed solve's refinement defect (double-float rows) on a smooth x
    # with b = 0: each row cancels to O(h^2) of s_i, so plain FP32 rows would
    # miss the bound
    xs = _smooth_field(info, disc)
    xs[:3 * nv] *= vmask
    refs, ss = sample_rows(box, H, L, disc, xs, rows, nu_a, with_abs=True)
    assert pb.refinement_residual_kind() == "df32"
    rd = pb.new_vector(L, prec=hhg.FP32)
    pb.refinement_residual(L, pb.to_device(L, xs), pb.new_vector(L), rd)
    gd = _gather(pb.to_host(L, rd), rows, nv)
    errd = np.abs(gd + refs)
    boundd = 2.0 ** -24 * np.abs(refs) + 2.0 ** -32 * ss
    assert np.all(errd <= boundd), float((errd / np.maximum(boundd, 1e-300)).max())
    assert np.median(np.abs(refs[~dirichlet]) / ss[~dirichlet]) < 1e-3
    del rd

    # FP32 apply and residual (the V-cycle precision; the benchmark's roofline kernel)
    x32 = x.astype(np.float32).astype(np.float64)
    b32 = b.astype(np.float32).astype(np.float64)
    ref32, s32 = sample_rows(box, H, L, disc, x32, rows, nu_a, with_abs=True)
    xd32 = pb.to_device(L, x32, prec=hhg.FP32)
    y32 = pb.new_vector(L, prec=hhg.FP32)
    pb.apply(L, "FULL", xd32, y32)
    got32 = _gather(pb.to_host(L, y32), rows, nv)
    err32 = np.abs(got32 - ref32)
    assert np.all(err32 <= 256 * EPS32 * s32), (float((err32 / np.maximum(s32, 1e-300)).max()), shapes[L])
    assert np.all(got32[dirichlet] == 0.0)
    r32 = pb.new_vector(L, prec=hhg.FP32)
    pb.residual(L, xd32, pb.to_device(L, b32, prec=hhg.FP32), r32)
    gr32 = _gather(pb.to_host(L, r32), rows, nv)
    b32row = _gather(b32, rows, nv)
    assert np.all(np.abs(gr32 - (b32row - ref32)) <= 256 * EPS32 * (s32 + np.abs(b32row)))


def test_fmg_headline_tuple_parity():
    """The benchmark's FMG (P2-P1, the paper's cube solution, coarse level 2,
    s = (1, 3, 1, 1, A_f, 3)) in FP64 at level 4 under autotuned launch
    shapes against the oracle's Algorithm 1: 1e-10 relative."""
    from hhg_inputs import Workload
    from oracle.stokes import Params, StokesHierarchy
    from paper_2010_13513_gb300 import hhg
    torch.cuda.set_stream(torch.cuda.Stream())
    wl = Workload("paper")
    L, lc = 4, 2
    s = dict(nu_pre=1, nu_post=3, nu_inc=1, kappa=1, ahat="f", xi=3, omega_inv=0.32)
    pb = hhg.Problem(hhg.Mesh.box(1, 1, 1, 1.0), disc="P2P1", L=L, coarse_level=lc, solve="fp64")
    hhg.set_workload_rhs(pb, wl)
    pb.autotune(reps=2)
    x = pb.new_vector(L)
    pb.fmg_solve(hhg.Params.make(**s), x)
    ref = StokesHierarchy((1, 1, 1), 1.0, L, "P2P1", coarse_level=lc, workload=wl).fmg(Params(**s))
    assert rel(pb.to_host(L, x), ref) < 1e-10


def test_batch_matches_oracle():
    """Every problem of a batch of uneven problems, solved by the batch's one
    graph, against the oracle's FMG of that problem: FP64 problems at 1e-10,
    mixed-precision problems within 1e-5 (FP32 V-cycles; no parity claim)."""
    from hhg_inputs import Workload
    from oracle.stokes import Params, StokesHierarchy
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    specs = [("P1P1", (1, 1, 1), 3, 0, "fp64"), ("P2P1", (2, 1, 1), 3, 1, "mixed"),
             ("P1P1", (1, 2, 2), 2, 0, "mixed"), ("P2P1", (1, 1, 1), 2, 1, "fp64")]
    om = {"P1P1": 0.5, "P2P1": 0.3}
    pbs, prms, refs = [], [], []
    with torch.cuda.stream(stream):
        for i, (disc, box, L, lc, solve) in enumerate(specs):
            H = 1.0 / max(box)
            wl = Workload("modes", seed=100 + i, box=box, H=H)
            pb = hhg.Problem(hhg.Mesh.box(*box, H), disc=disc, L=L, coarse_level=lc, solve=solve)
            hhg.set_workload_rhs(pb, wl)
            s = dict(nu_pre=1, nu_post=2, nu_inc=1, kappa=1, ahat="f", xi=2, omega_inv=om[disc])
            prms.append(hhg.Params.make(**s))
            pbs.append(pb)
            refs.append(StokesHierarchy(box, H, L, disc, coarse_level=lc, workload=wl).fmg(Params(**s)))
        batch = hhg.Batch(pbs)
        batch.fmg_solve(prms, stream)
        stream.synchronize()
    for (disc, box, L, lc, solve), pb, ref in zip(specs, pbs, refs):
        got = pb.to_host(L, pb.level_vector(L, "x"))
        assert rel(got, ref) < (1e-10 if solve == "fp64" else 1e-5), (disc, box, L, solve, rel(got, ref))
