"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  The aim is that a plausible mistake
anywhere in the oracle (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from hhg_inputs import Workload, kuhn_box_macro_mesh
from oracle import fe, workmodel
from oracle.mesh import Lattice, bey_refine
from oracle.stokes import Params, StokesHierarchy, StokesLevel, prolongation_matrix

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# --------------------------------------------------------------------------
# work-unit model: Table 3 and the worked example of Sec. 4.2
# --------------------------------------------------------------------------
def test_work_units_table3():
    g = _load("table3_work_units.json")
    for e in g["entries"]:
        s = e["s"]
        wu = float(workmodel.fmg_work(e["disc"], *s))
        assert round(wu, e["digits"]) == pytest.approx(e["wu"], abs=1e-12), (e, wu)


def test_work_unit_normalisations():
    g = _load("table3_work_units.json")["normalized"]
    from fractions import Fraction as F
    a, b, c = workmodel.normalized_blocks("P2P1")
    assert (a, b, c) == (F(*g["P2P1_A"]), F(*g["P2P1_B"]), 0)
    a, b, c = workmodel.normalized_blocks("P1P1")
    assert (a, b, c) == (F(*g["P1P1_A"]), F(*g["P1P1_B"]), F(*g["P1P1_C"]))
    assert workmodel.relaxation_work("P2P1", "f", 1) == F(*g["P2P1_uzawa_Af_xi1"])
    assert workmodel.relaxation_work("P2P1", "s", 1) == F(*g["P2P1_uzawa_As_xi1"])
    # finite-level normalisations approach the limit
    a6 = workmodel.normalized_blocks("P2P1", 12)[0]
    assert abs(float(a6) - 46 / 72) < 2e-3


def test_asymptotic_ratios():
    g = _load("table3_work_units.json")["asymptotic_ratios"]
    from fractions import Fraction as F
    assert workmodel.unknown_ratio_limit() == F(*g["unknowns"])
    # leading-order ratios of Eq. wu-comparison-p2p1-p1p1 from the level formulas
    l = 14
    wa2, wb2, _ = workmodel.block_work("P2P1", l)
    wa1, wb1, wc1 = workmodel.block_work("P1P1", l + 1)
    assert abs(wa2 / wa1 - 23 / 12) < 1e-3
    assert abs(wb2 / wb1 - 13 / 24) < 1e-3
    assert abs((wa2 + 2 * wb2) / (wa1 + 2 * wb1 + wc1) - 9 / 10) < 1e-3


# --------------------------------------------------------------------------
# mesh: Bey refinement, Table 1 counts, P2(l) = P1(l+1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("level", [1, 2, 3])
def test_bey_refinement_is_kuhn_lattice(level):
    verts, tets = kuhn_box_macro_mesh(1, 1, 1)
    bey = {frozenset(t) for t in bey_refine(verts, tets, level)}
    lat = Lattice((1, 1, 1), 1.0, level)
    T, _ = lat.tets()
    kuhn = {frozenset(tuple(float(c) for c in v * lat.h) for v in t) for t in T}
    assert len(bey) == 6 * 8 ** level
    assert bey == kuhn


def _group_counts(level):
    """Inner and closure counts of each DoF group in the macro tetrahedron
    2n >= P0 >= P1 >= P2 >= 0 of the doubled lattice."""
    n = 2 ** level
    out = {}
    rng = range(0, 2 * n + 1)
    for o in itertools.product((0, 1), repeat=3):
        inner = closure = 0
        for P in itertools.product(rng, repeat=3):
            if tuple(p % 2 for p in P) != o:
                continue
            if 2 * n >= P[0] >= P[1] >= P[2] >= 0:
                closure += 1
                if 2 * n > P[0] > P[1] > P[2] > 0:
                    inner += 1
        out[o] = (inner, closure)
    return out


@pytest.mark.parametrize("level", [2, 3, 4])
def test_table1_unknown_counts(level):
    n = 2 ** level
    N = workmodel.n_tet
    counts = _group_counts(level)
    assert counts[(0, 0, 0)] == (N(n - 3), N(n + 1))
    edges = sorted(v for o, v in counts.items() if o != (0, 0, 0))
    expect = sorted([(N(n - 1), N(n - 1))] + [(N(n - 2), N(n))] * 6)
    assert edges == expect
    t1 = workmodel.table1_counts(level)
    assert t1["vertices"] == (N(n - 3), N(n + 1))


def _refined_mesh_counts(verts, tets, level):
    """(vertices, edges, faces, tetrahedra, boundary faces, volume) of the
    macro mesh refined `level` times by Bey's rule; points keyed on the
    dyadic grid of spacing 2^-(level+2), faces with the number of
    tetrahedra that share them."""
    kids = bey_refine(verts, tets, level)
    s = 2.0 ** (level + 2)
    key = lambda x: tuple(int(round(c * s)) for c in x)
    V, E, F = set(), set(), {}
    vol = 0.0
    for t in kids:
        ks = [key(x) for x in t]
        V.update(ks)
        E.update(frozenset((ks[a], ks[b])) for a in range(4) for b in range(a + 1, 4))
        for f in itertools.combinations(ks, 3):
            F[frozenset(f)] = F.get(frozenset(f), 0) + 1
        X = np.array(t)
        vol += abs(np.linalg.det(X[1:] - X[0])) / 6.0
    assert set(F.values()) <= {1, 2}                       # conforming: a face is shared by at most two
    return len(V), len(E), len(F), len(kids), sum(1 for m in F.values() if m == 1), vol


def test_cube24_refinement_counts_and_paper_unknowns():
    """The cube of 24 macro tetrahedra of Sec. 5.1.1 (corners, face centres,
    centre): Bey refinement (Sec. 2) gives conforming meshes of volume 1
    whose vertex, edge, face and tetrahedron counts follow uniform refinement
    (every edge gets a midpoint, every face three inner edges and four faces,
    every tetrahedron one inner edge, eight inner faces and eight children),
    and continuing those counts to the paper's levels gives the unknowns it
    quotes: about 4.3e6 for P1-P1 at L = 6 (four fields on the vertices) and
    about 3.4e6 for P2-P1 at L = 5 (velocity on the level-6 vertices, which are
    the level-5 P2 nodes, pressure on the level-5 vertices)."""
    from hhg_inputs import cube24_macro_mesh
    verts, tets = cube24_macro_mesh()
    V, E, F, T = 15, 50, 60, 24
    counts = [(V, E, F, T)]
    for _ in range(6):
        V, E, F, T = V + E, 2 * E + 3 * F + T, 4 * F + 8 * T, 8 * T
        counts.append((V, E, F, T))
    for level in (0, 1, 2):
        v, e, f, t, fb, vol = _refined_mesh_counts(verts, tets, level)
        assert (v, e, f, t) == counts[level]
        assert fb == 24 * 4 ** level                        # the cube's 6 faces, 4 triangles each
        assert v - e + f - t == 1                           # Euler characteristic of a ball
        assert vol == pytest.approx(1.0, rel=1e-12)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "cube24_unknowns.json")))
    p1 = 4 * counts[6][0]
    p2 = 3 * counts[6][0] + counts[5][0]
    assert (p1, p2) == (4293636, 3357572)
    assert round(p1, -5) == gold["P1P1_L6_about"] and round(p2, -5) == gold["P2P1_L5_about"]


@pytest.mark.parametrize("disc,box,H", [("P1P1", (1, 1, 1), 1.0), ("P2P1", (1, 1, 1), 1.0),
                                        ("P1P1", (2, 1, 1), 0.5), ("P2P1", (1, 2, 1), 0.5)])
def test_unstructured_assembly_equals_lattice_on_kuhn_boxes(disc, box, H):
    """The element-by-element assembly on a Bey-refined macro mesh
    (oracle/unstructured.py, no lattice) and the lattice assembly
    (StokesLevel) give the same blocks, masses and Dirichlet nodes on Kuhn
    boxes, entry by entry: two independent paths to Eq. stokes-discrete."""
    from oracle.unstructured import UnstructuredLevel
    verts, tets = kuhn_box_macro_mesh(*box, H)
    u = UnstructuredLevel(verts, tets, 2, disc)
    lev = StokesLevel(box, H, 2, disc)
    assert (u.nv, u.np) == (lev.nv, lev.np)
    for a, b in [(u.A, lev.A), (u.Mv, lev.Mv), (u.C, lev.C), (u.Mp, lev.Mp_full)] + list(zip(u.B, lev.B)):
        scale = max(abs(b).max(), 1e-300)
        assert abs(a - b).max() <= 1e-13 * scale
    assert np.array_equal(u.vbnd, lev.vbnd)
    x = np.random.default_rng(5).uniform(-1, 1, lev.size)
    x[:3 * lev.nv] *= np.tile(lev.vint, 3)
    assert np.allclose(u.apply(x), lev.apply(x), rtol=0, atol=1e-13 * np.abs(lev.apply(x)).max())


@pytest.mark.parametrize("disc,level", [("P1P1", 2), ("P2P1", 1)])
def test_unstructured_operators_on_cube24(disc, level):
    """Eq. stokes-discrete on the paper's cube of 24 macro tetrahedra (not a
    Kuhn box): node counts of the refinement (P2 nodes = next level's
    vertices), Dirichlet nodes = the nodes on the cube's surface, masses
    integrating to the volume, A and C symmetric with zero row sums, A
    annihilating linear fields at interior nodes and reproducing -Laplace(q)
    for a quadratic q with P2, and the divergence blocks exact on linear
    (P1) or quadratic (P2) velocities: (B_d u)_k = -int psi_k d_d u."""
    from hhg_inputs import cube24_macro_mesh
    from oracle.unstructured import UnstructuredLevel
    verts, tets = cube24_macro_mesh()
    u = UnstructuredLevel(verts, tets, level, disc)
    V = [15, 65, 369, 2465]
    assert u.np == V[level] and u.nv == (V[level] if disc == "P1P1" else V[level + 1])
    on_surface = lambda P: np.any((np.abs(P) < 1e-12) | (np.abs(P - 1.0) < 1e-12), axis=1)
    assert np.array_equal(u.vbnd, on_surface(u.vcoords))
    one_v, one_p = np.ones(u.nv), np.ones(u.np)
    assert one_v @ (u.Mv @ one_v) == pytest.approx(1.0, rel=1e-13)
    assert one_p @ (u.Mp @ one_p) == pytest.approx(1.0, rel=1e-13)
    for M, one in ((u.A, one_v), (u.C, one_p)):
        size = max(abs(M).max(), 1e-300)
        assert abs(M - M.T).max() <= 1e-14 * size
        assert np.abs(M @ one).max() <= 1e-12 * size
    X, Y, Z = u.vcoords.T
    Xp = u.pcoords
    lin = 0.3 * X - 0.7 * Y + 1.1 * Z
    assert np.abs((u.A @ lin)[u.vint]).max() <= 1e-12 * abs(u.A).max()
    if disc == "P2P1":
        q = X * X + 2 * Y * Y - Z * Z + X * Y                   # Laplace q = 2 + 4 - 2 = 4
        ref = -4.0 * (u.Mv @ one_v)
        assert np.abs((u.A @ q - ref)[u.vint]).max() <= 1e-12 * np.abs(ref).max()
    xp, yp, zp = Xp.T
    for d, coord in enumerate((X, Y, Z)):
        if disc == "P1P1":
            # u_d = coordinate d: div u = 1
            assert np.allclose(u.B[d] @ coord, -(u.Mp @ one_p), rtol=0, atol=1e-13)
        else:
            # u_d = coordinate d squared: div u = 2 x_d, linear, so the P1 pressure mass is exact
            pd = (xp, yp, zp)[d]
            assert np.allclose(u.B[d] @ (coord * coord), -2.0 * (u.Mp @ pd), rtol=0, atol=1e-13)


@pytest.mark.parametrize("level", [1, 2, 3])
def test_p2_nodes_equal_p1_next_level(level):
    a = Lattice((1, 1, 1), 1.0, level)
    b = Lattice((1, 1, 1), 1.0, level + 1)
    assert a.p2_count() == b.p1_count()
    assert np.allclose(a.p2_coords(), b.p1_coords())


# --------------------------------------------------------------------------
# stencil structure: Table 2 and the 15-point P1 stencil
# --------------------------------------------------------------------------
def _pattern(lev):
    nt = lev.tet_vdofs.shape[0]
    r = np.repeat(lev.tet_vdofs[:, :, None], lev.tet_vdofs.shape[1], axis=2).ravel()
    c = np.repeat(lev.tet_vdofs[:, None, :], lev.tet_vdofs.shape[1], axis=1).ravel()
    return sp.coo_matrix((np.ones(r.size), (r, c)), shape=(lev.nv, lev.nv)).tocsr()


def test_table2_stencil_sizes():
    g = _load("tables_1_2_counts.json")["table2"]
    lev = StokesLevel((1, 1, 1), 1.0, 3, "P2P1")
    pat = _pattern(lev)
    lat = lev.lat
    IJK = lat.p2_int_coords()
    is_vertex = np.all(IJK % 2 == 0, axis=1)
    centre = np.array([8, 8, 8])             # a point deep inside (doubled lattice, n = 8)
    from_all, from_vertex = {}, {}
    for o in itertools.product((0, 1), repeat=3):
        P = centre + np.array(o)
        i = lat.p2_index(P)
        cols = pat.indices[pat.indptr[i]:pat.indptr[i + 1]]
        from_all[o] = len(cols)
        from_vertex[o] = int(is_vertex[cols].sum())
    assert from_all[(0, 0, 0)] == g["vertex_from_all"]
    assert from_vertex[(0, 0, 0)] == g["vertex_from_vertex"]
    edges = [o for o in from_all if o != (0, 0, 0)]
    assert sorted(from_all[o] for o in edges) == sorted(g["edges_from_all"])
    assert sorted(from_vertex[o] for o in edges) == sorted(g["edges_from_vertex"])
    # an edge row with 27 entries has 8 vertex neighbours, one with 19 has 6
    for o in edges:
        assert (from_all[o], from_vertex[o]) in ((27, 8), (19, 6))


def test_p1_fifteen_point_stencil():
    lev = StokesLevel((1, 1, 1), 1.0, 3, "P1P1")
    pat = _pattern(lev)
    i = lev.lat.p1_index(np.array([4, 4, 4]))
    assert pat.indptr[i + 1] - pat.indptr[i] == 15


# --------------------------------------------------------------------------
# element matrices and stencil values: closed forms
# --------------------------------------------------------------------------
def _random_tet(seed):
    rng = np.random.default_rng(seed)
    while True:
        X = rng.uniform(-1, 1, size=(4, 3))
        if abs(np.linalg.det(X[1:] - X[0])) > 0.1:
            return X


def test_element_p1_closed_forms():
    X = _random_tet(0)
    vol, g = fe.tet_geometry(X)
    M = fe.mass(X, 1)
    assert np.allclose(M, vol / 20 * (np.ones((4, 4)) + np.eye(4)), rtol=1e-13)
    K = fe.stiffness(X, 1)
    assert np.allclose(K, vol * g @ g.T, rtol=1e-12)
    assert np.allclose(K.sum(axis=1), 0, atol=1e-12)


@pytest.mark.parametrize("order", [1, 2])
def test_element_matrices_against_quadrature(order):
    """Exact barycentric integration against an independent fine product
    quadrature of the collapsed cube (degree <= 4 integrands)."""
    X = _random_tet(3)
    vol, g = fe.tet_geometry(X)
    xg, wg = np.polynomial.legendre.leggauss(6)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    pts, wts = [], []
    for a, wa in zip(xg, wg):
        for b, wb in zip(xg, wg):
            for c, wc in zip(xg, wg):
                r = np.array([a, (1 - a) * b, (1 - a) * (1 - b) * c])
                pts.append(r)
                wts.append(wa * wb * wc * (1 - a) ** 2 * (1 - b))
    pts, wts = np.array(pts), np.array(wts) * 6 * vol
    lmb = np.concatenate([1 - pts.sum(axis=1, keepdims=True), pts], axis=1)
    phi = fe.basis_values(lmb, order)
    M = (phi * wts[:, None]).T @ phi
    assert np.allclose(M, fe.mass(X, order), rtol=1e-11, atol=1e-14)
    # gradients by central differences of the basis in barycentric space
    eps = 1e-6
    grads = np.zeros((len(pts), phi.shape[1], 3))
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)
    for d in range(3):
        dx = np.zeros(3)
        dx[d] = eps
        dl = np.linalg.solve(J, dx)
        lp = lmb + np.concatenate([[-dl.sum()], dl])[None, :]
        lm = lmb - np.concatenate([[-dl.sum()], dl])[None, :]
        grads[:, :, d] = (fe.basis_values(lp, order) - fe.basis_values(lm, order)) / (2 * eps)
    K = np.einsum("q,qad,qbd->ab", wts, grads, grads)
    assert np.allclose(K, fe.stiffness(X, order), rtol=1e-6, atol=1e-8)
    D = fe.divergence(X, order)
    for d in range(3):
        Dq = -np.einsum("q,qk,qj->kj", wts, lmb, grads[:, :, d])
        assert np.allclose(Dq, D[d], rtol=1e-6, atol=1e-8)


def test_p1_laplacian_is_seven_point():
    """On the Kuhn lattice the P1 Laplacian reduces to h (6, -1 x 6)."""
    lev = StokesLevel((1, 1, 1), 1.0, 3, "P1P1")
    h = lev.lat.h
    i = lev.lat.p1_index(np.array([4, 4, 4]))
    row = lev.A.getrow(i).toarray().ravel()
    nz = np.nonzero(np.abs(row) > 1e-14)[0]
    assert len(nz) == 7
    assert row[i] == pytest.approx(6 * h, rel=1e-13)
    for d in [(1, 0, 0), (0, 1, 0), (0, 0, 1)]:
        for s in (1, -1):
            j = lev.lat.p1_index(np.array([4, 4, 4]) + s * np.array(d))
            assert row[j] == pytest.approx(-h, rel=1e-13)
    assert lev.ML[i] == pytest.approx(h ** 3, rel=1e-13)
    # PSPG: delta h_T^2 times the Laplacian stencil, h_T = (h^3/6)^(1/3)
    crow = lev.C.getrow(i).toarray().ravel()
    hT2 = (h ** 3 / 6) ** (2 / 3)
    assert np.allclose(crow, row * hT2 / 12.0, rtol=1e-12, atol=1e-18)


@pytest.mark.parametrize("disc", ["P1P1", "P2P1"])
def test_operator_invariants(disc):
    lev = StokesLevel((1, 1, 1), 1.0, 2, disc)
    I = np.nonzero(lev.vint)[0]
    A = lev.A
    assert abs(A - A.T).max() < 1e-15
    assert abs(lev.C - lev.C.T).max() < 1e-18
    assert abs(lev.Mv - lev.Mv.T).max() < 1e-18
    rs = np.asarray(A.sum(axis=1)).ravel()[I]
    assert np.all(np.abs(rs) <= 1e-14 * np.abs(A).sum(axis=1).A.ravel()[I] + 1e-16)
    assert np.allclose(lev.C @ np.ones(lev.np), 0, atol=1e-15)
    assert lev.Mv.sum() == pytest.approx(1.0, rel=1e-13)
    assert lev.Mp.sum() == pytest.approx(1.0, rel=1e-13)
    # B^T 1 = 0 on interior velocity rows (grad of a constant pressure)
    for c in range(3):
        assert np.allclose((lev.B[c].T @ np.ones(lev.np))[I], 0, atol=1e-15)


@pytest.mark.parametrize("disc", ["P1P1", "P2P1"])
def test_divergence_closed_form(disc):
    """(B I u)_k = -int psi_k div u for polynomial u of the velocity degree."""
    lev = StokesLevel((1, 1, 1), 1.0, 2, disc)
    Xv, Xp = lev.vcoords(), lev.pcoords()
    if disc == "P1P1":
        Gm = np.array([[0.3, -1.2, 0.5], [2.0, 0.1, -0.7], [0.4, 0.9, -1.6]])
        u = Xv @ Gm.T + np.array([0.1, -0.2, 0.3])
        div = np.trace(Gm)
        Bu = sum(lev.B[c] @ u[:, c] for c in range(3))
        assert np.allclose(Bu, -div * lev.ML, rtol=1e-12, atol=1e-15)
    else:
        x, y, z = Xv[:, 0], Xv[:, 1], Xv[:, 2]
        u = np.stack([x * x + y * z, x * y - z * z, 2 * x * z + y * y], axis=1)
        dx, dy, dz = Xp[:, 0], Xp[:, 1], Xp[:, 2]
        divp = 2 * dx + dx + 2 * dx                # d/dx(x^2) + d/dy(xy) + d/dz(2xz)
        Bu = sum(lev.B[c] @ u[:, c] for c in range(3))
        assert np.allclose(Bu, -(lev.Mp @ divp), rtol=1e-11, atol=1e-14)


def test_p2_laplacian_closed_form():
    """(A I q)_i = -Delta q int phi_i at interior nodes for quadratic q."""
    lev = StokesLevel((1, 1, 1), 1.0, 2, "P2P1")
    X = lev.vcoords()
    q = 1.5 * X[:, 0] ** 2 - 0.5 * X[:, 1] ** 2 + 2 * X[:, 2] ** 2 + X[:, 0] * X[:, 1] - X[:, 2]
    lap = 3.0 - 1.0 + 4.0
    intphi = np.asarray(lev.Mv.sum(axis=1)).ravel()
    Aq = lev.A @ q
    I = lev.vint
    assert np.allclose(Aq[I], -lap * intphi[I], rtol=1e-11, atol=1e-14)


# --------------------------------------------------------------------------
# brute force: vectorised assembly against a plain per-element loop
# --------------------------------------------------------------------------
@pytest.mark.parametrize("disc", ["P1P1", "P2P1"])
def test_assembly_brute_force(disc):
    lev = StokesLevel((1, 2, 1), 0.5, 1, disc, nu_a=1.3)
    lat = lev.lat
    T, _ = lat.tets()
    A = np.zeros((lev.nv, lev.nv))
    Bx = np.zeros((lev.np, lev.nv))
    C = np.zeros((lev.np, lev.np))
    for t in range(T.shape[0]):
        X = T[t].astype(float) * lat.h
        nu = math.exp(1.3 * X[:, 2].mean())
        vd, pd = lev.tet_vdofs[t], lev.tet_pdofs[t]
        K = fe.stiffness(X, lev.order_v) * nu
        D = fe.divergence(X, lev.order_v)[0]
        for a in range(len(vd)):
            for b in range(len(vd)):
                A[vd[a], vd[b]] += K[a, b]
        for k in range(4):
            for b in range(len(vd)):
                Bx[pd[k], vd[b]] += D[k, b]
        if disc == "P1P1":
            Ce = fe.pspg(X) / nu
            for k in range(4):
                for l in range(4):
                    C[pd[k], pd[l]] += Ce[k, l]
    assert np.allclose(lev.A.toarray(), A, rtol=1e-13, atol=1e-15)
    assert np.allclose(lev.B[0].toarray(), Bx, rtol=1e-13, atol=1e-15)
    assert np.allclose(lev.C.toarray(), C, rtol=1e-13, atol=1e-17)


# --------------------------------------------------------------------------
# Gauss-Seidel ordering
# --------------------------------------------------------------------------
@pytest.mark.parametrize("disc", ["P1P1", "P2P1"])
def test_colour_phases_are_uncoupled_and_cover(disc):
    lev = StokesLevel((1, 1, 1), 1.0, 2, disc)
    pat = _pattern(lev)
    allidx = np.concatenate(lev.phases)
    assert len(allidx) == len(set(allidx.tolist())) == int(lev.vint.sum())
    for S in lev.phases:
        sub = pat[S][:, S].tocoo()
        assert np.all(sub.row == sub.col)
    assert len(lev.phases) == (4 if disc == "P1P1" else 11)


@pytest.mark.parametrize("disc", ["P1P1", "P2P1"])
def test_gs_sweep_equals_triangular_solve(disc):
    """A forward sweep is (D + L_pi)^{-1} (b - U_pi x) under the phase
    permutation pi; a backward sweep uses the reversed permutation."""
    lev = StokesLevel((1, 1, 1), 1.0, 2, disc)
    pi = np.concatenate(lev.phases)
    Ad = lev.A.toarray()[np.ix_(pi, pi)]
    rng = np.random.default_rng(5)
    b = np.zeros(lev.nv)
    b[pi] = rng.uniform(-1, 1, len(pi))
    x0 = np.zeros(lev.nv)
    x0[pi] = rng.uniform(-1, 1, len(pi))
    x = x0.copy()
    lev.gs_sweep(x, b)
    Lw = np.tril(Ad)
    U = np.triu(Ad, 1)
    ref = np.linalg.solve(Lw, b[pi] - U @ x0[pi])
    assert np.allclose(x[pi], ref, rtol=1e-12, atol=1e-13)
    x = x0.copy()
    lev.gs_sweep(x, b, backward=True)
    ref = np.linalg.solve(np.triu(Ad), b[pi] - np.tril(Ad, -1) @ x0[pi])
    assert np.allclose(x[pi], ref, rtol=1e-12, atol=1e-13)


# --------------------------------------------------------------------------
# transfers
# --------------------------------------------------------------------------
def test_prolongation_reproduces_polynomials():
    fine = Lattice((2, 1, 1), 0.5, 2)
    coarse = Lattice((2, 1, 1), 0.5, 1)
    P1 = prolongation_matrix(fine, coarse, 1)
    lin = lambda X: 0.3 + X[:, 0] - 2 * X[:, 1] + 0.7 * X[:, 2]
    assert np.allclose(P1 @ lin(coarse.p1_coords()), lin(fine.p1_coords()), atol=1e-14)
    P2 = prolongation_matrix(fine, coarse, 2)
    quad = lambda X: 1 + X[:, 0] * X[:, 1] - 3 * X[:, 2] ** 2 + X[:, 0] - 0.5 * X[:, 1] * X[:, 2]
    assert np.allclose(P2 @ quad(coarse.p2_coords()), quad(fine.p2_coords()), atol=1e-13)
    # a quadratic is not reproduced by linear interpolation (the pin is not vacuous)
    assert not np.allclose(P1 @ quad(coarse.p1_coords()), quad(fine.p1_coords()), atol=1e-6)
    # rows are partitions of unity
    assert np.allclose(P2.sum(axis=1), 1) and np.allclose(P1.sum(axis=1), 1)


# --------------------------------------------------------------------------
# coarse solve, Uzawa invariants, multigrid convergence
# --------------------------------------------------------------------------
@pytest.mark.parametrize("disc,lc", [("P1P1", 0), ("P1P1", 1), ("P2P1", 1)])
def test_coarse_solve(disc, lc):
    hy = StokesHierarchy((1, 1, 1), 1.0, lc, disc, coarse_level=lc, workload=Workload("curl"))
    lev = hy.lv[lc]
    b = hy.rhs[lc]
    x = hy.coarse_solve(b)
    r = lev.residual(x, b)
    assert max(lev.norms(r)) <= 1e-12 * max(1.0, max(lev.norms(b)))
    _, p = lev.split(x)
    assert abs(np.dot(lev.ML, p)) < 1e-13


def test_uzawa_preserves_pressure_mean_and_rhs_compatible():
    hy = StokesHierarchy((1, 1, 1), 1.0, 3, "P1P1", workload=Workload("curl"))
    lev = hy.lv[3]
    b = hy.rhs[3]
    _, g = lev.split(b)
    assert abs(g.sum()) < 1e-14 * np.abs(g).sum()
    rng = np.random.default_rng(2)
    x = rng.uniform(-1, 1, lev.size)
    x[:3 * lev.nv] *= np.tile(lev.vint, 3)
    m0 = np.dot(lev.ML, lev.split(x)[1])
    x1 = lev.uzawa(x, b, Params(ahat="s", xi=2, omega_inv=0.6))
    assert np.dot(lev.ML, lev.split(x1)[1]) == pytest.approx(m0, abs=1e-13)


@pytest.mark.parametrize("disc,L,lc,rate", [("P1P1", 3, 0, 0.35), ("P2P1", 3, 1, 0.75)])
def test_vcycle_contracts(disc, L, lc, rate):
    hy = StokesHierarchy((1, 1, 1), 1.0, L, disc, coarse_level=lc, workload=Workload("curl"))
    lev = hy.lv[L]
    b = hy.rhs[L]
    prm = Params(2, 2, 1, 1, "f", 3, 0.4 if disc == "P2P1" else 0.6)
    x = np.zeros(lev.size)
    r0 = max(lev.norms(b))
    for _ in range(6):
        x = lev.project_pressure(hy.vcycle(L, L, x, b, prm))
    r6 = max(lev.norms(lev.residual(x, b)))
    assert r6 < rate ** 6 * r0


# --------------------------------------------------------------------------
# discretisation orders (settles the rhs readings) and omega
# --------------------------------------------------------------------------
@pytest.mark.slow
def test_velocity_convergence_orders():
    errs = {}
    for disc, levels, lc in [("P1P1", (2, 3, 4), 0), ("P2P1", (2, 3), 1)]:
        for L in levels:
            hy = StokesHierarchy((1, 1, 1), 1.0, L, disc, coarse_level=lc, workload=Workload("curl"))
            om = 0.25 if disc == "P2P1" else 0.4
            x, it = hy.solve_to_tolerance(Params(2, 2, 1, 1, "f", 3, om), max_cycles=400)
            assert it < 400
            errs[(disc, L)] = hy.error_norms(x)
    s1 = math.log2(errs[("P1P1", 3)][0] / errs[("P1P1", 4)][0])
    s2 = math.log2(errs[("P2P1", 2)][0] / errs[("P2P1", 3)][0])
    assert 1.8 < s1 < 2.3, s1
    assert 2.7 < s2 < 3.4, s2
    sp1 = math.log2(errs[("P1P1", 3)][1] / errs[("P1P1", 4)][1])
    assert sp1 > 1.0


def test_variable_viscosity_reduces_to_constant():
    a = StokesLevel((1, 1, 1), 1.0, 2, "P1P1", nu_a=0.0)
    b = StokesLevel((1, 1, 1), 1.0, 2, "P1P1", nu_a=1e-300)
    assert abs(a.A - b.A).max() < 1e-15
    c = StokesLevel((1, 1, 1), 1.0, 2, "P1P1", nu_a=2.0)
    # nu >= 1 everywhere: the diagonal grows, C shrinks
    assert np.all(c.A.diagonal() >= a.A.diagonal() - 1e-15)
    assert np.all(np.abs(c.C.diagonal()) <= np.abs(a.C.diagonal()) + 1e-18)


@pytest.mark.slow
def test_variable_viscosity_order():
    nu_a = 1.5
    errs = []
    for L in (2, 3):
        hy = StokesHierarchy((1, 1, 1), 1.0, L, "P1P1", nu_a=nu_a, workload=Workload("curl", nu_a=nu_a))
        x, _ = hy.solve_to_tolerance(Params(2, 2, 1, 1, "f", 3, 0.6), max_cycles=400)
        errs.append(hy.error_norms(x)[0])
    assert 1.6 < math.log2(errs[0] / errs[1]) < 2.5


def test_omega_estimate_near_paper():
    """Loose pin of the S_hat = omega^{-1} M_L reading: the P1-P1 estimate on
    the 6-tetrahedron cube lands within 10 % of the paper's 0.570751 (which
    is for a 24-tetrahedron cube on level 6)."""
    ref = _load("tables_1_2_counts.json")["omega_inv"]["P1P1_L6"]
    hy = StokesHierarchy((1, 1, 1), 1.0, 4, "P1P1", workload=Workload("curl"))
    v0 = np.random.default_rng(0).uniform(-1, 1, hy.lv[4].np)
    om = hy.estimate_omega_inv(v0, iters=100)
    assert abs(om / ref - 1) < 0.10, om


@pytest.mark.parametrize("disc,nu_a", [("P1P1", 0.0), ("P2P1", 0.0), ("P1P1", 1.3), ("P2P1", 0.7)])
def test_sampled_rows_match_assembled(disc, nu_a):
    """The single-row evaluator used at full problem sizes equals the
    assembled operator (its own element loop, Eq. stokes-discrete)."""
    from oracle.sampled import sample_rows
    lev = StokesLevel((1, 2, 1), 0.5, 2, disc, nu_a=nu_a)
    x = np.random.default_rng(0).uniform(-1, 1, lev.size)
    y = lev.apply(x * np.concatenate([np.tile(lev.vint, 3), np.ones(lev.np)]))
    rng = np.random.default_rng(1)
    rows = [(int(f), int(rng.integers(0, lev.nv if f < 3 else lev.np))) for f in rng.integers(0, 4, 80)]
    xs = x * np.concatenate([np.tile(lev.vint, 3), np.ones(lev.np)])
    ys, ya = sample_rows((1, 2, 1), 0.5, 2, disc, xs, rows, nu_a, with_abs=True)
    ref = np.array([y[f * lev.nv + n] if f < 3 else y[3 * lev.nv + n] for f, n in rows])
    assert np.all(np.abs(ys - ref) <= 1e-14 * (ya + 1e-300) + 1e-300)


def test_mlp_gradients_match_finite_differences():
    """Back-propagation of the learned-coarse-correction MLP against central
    differences of the loss (the definition of the derivative)."""
    from oracle import mlp
    rng = np.random.default_rng(3)
    n, H, B = 7, 9, 5
    params = mlp.init(n, H, seed=1)
    params = [p + 0.05 * rng.standard_normal(p.shape) for p in params]
    X = rng.standard_normal((B, n))
    T = rng.standard_normal((B, n))
    g = mlp.grads(params, X, T)
    eps = 1e-6
    for pi, p in enumerate(params):
        flat = p.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = mlp.loss(params, X, T)
            flat[idx] = old - eps
            lm = mlp.loss(params, X, T)
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            assert abs(fd - g[pi].reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(fd)), (pi, idx)


@pytest.mark.parametrize("disc,L", [("P1P1", 2), ("P2P1", 1), ("P2P1", 2)])
def test_paper_gs_order_is_textbook_gauss_seidel(disc, L):
    """The oracle's 'paper' Gauss-Seidel order (Sec. 5.2: one kernel per DoF
    group, the vertex DoFs in lexicographic order, then each edge group)
    equals the textbook loop u_i <- (f_i - sum_{j != i} a_ij u_j) / a_ii over
    the interior DoFs one at a time in that order, forward and backward --
    which also checks that an edge group can be updated at once."""
    from oracle.stokes import StokesLevel
    lev = StokesLevel((1, 1, 1), 1.0, L, disc)
    lev.set_gs_order("paper")
    rng = np.random.default_rng(11)
    u0 = np.where(lev.vint, rng.standard_normal(lev.nv), 0.0)
    rhs = rng.standard_normal(lev.nv)
    A = lev.A.toarray()
    if disc == "P1P1":
        vert = np.ones(lev.nv, dtype=bool)
    else:
        vert = np.all(lev.lat.p2_int_coords() % 2 == 0, axis=1)
    order = [int(i) for i in np.nonzero(lev.vint & vert)[0]]          # ascending node number = lexicographic
    for S in lev.phases[4:]:
        order += [int(i) for i in S]
    want = {}
    for backward in (False, True):
        w = u0.copy()
        for i in (order[::-1] if backward else order):
            w[i] = (rhs[i] - A[i] @ w + A[i, i] * w[i]) / A[i, i]
        got = u0.copy()
        lev.gs_sweep(got, rhs, backward=backward)
        assert np.abs(got - w).max() <= 1e-12 * np.abs(w).max(), backward
        want[backward] = w
    # with more than one interior vertex the multicolour order is a
    # different sweep (same fixed point)
    mc = u0.copy()
    lev.set_gs_order("multicolour")
    lev.gs_sweep(mc, rhs)
    if np.count_nonzero(lev.vint & vert) > 1:
        assert np.abs(mc - want[False]).max() > 1e-6


# --------------------------------------------------------------------------
# closed-form pins of the error norms (Eq. error), the omega^{-1} power
# iteration (Eq. omega-eigenvalue-problem) and the Uzawa pressure update
# --------------------------------------------------------------------------
class _PolyWorkload:
    """Polynomial exact solution with zero Dirichlet data (only exact_* and
    the rhs hooks the hierarchy calls are needed)."""

    def __init__(self, u, p):
        self.u, self.p = u, p

    def forcing(self, X):
        return np.zeros((X.shape[0], 3))

    def dirichlet(self, X):
        return np.zeros((X.shape[0], 3))

    def exact_velocity(self, X):
        return self.u(X)

    def exact_pressure(self, X):
        return self.p(X)


def test_lattice_index_inverse():
    lat = Lattice((2, 1, 3), 0.5, 2)
    for idx in (0, 7, lat.p1_count() - 1, 123):
        assert np.array_equal(lat.p1_int_coords_of(idx), lat.p1_int_coords()[idx])
    for idx in (0, 11, lat.p2_count() - 1, 2345):
        assert np.array_equal(lat.p2_int_coords_of(idx), lat.p2_int_coords()[idx])


@pytest.mark.parametrize("disc", ["P1P1", "P2P1"])
def test_error_norms_closed_forms(disc):
    """Eq. error with x = 0 is the M-norm of the exact fields on level l+1.
    The consistent mass matrix integrates the interpolant exactly, so for
    u* = (x, 0, 0) (P1) or (x^2, 0, 0) (P2) the velocity part is sqrt(1/3)
    or sqrt(1/5), and for p* = x the mean-zero pressure part is
    ||x - 1/2||_L2 = sqrt(1/12) (sqrt(1/3) if the mean were not removed; a
    lumped mass gives neither).  With x = the interpolant of (u*, p*) on
    level l, I x reproduces the polynomials and both parts vanish."""
    if disc == "P1P1":
        u = lambda X: np.stack([X[:, 0], 0 * X[:, 0], 0 * X[:, 0]], axis=1)
        ref_u = math.sqrt(1.0 / 3.0)
    else:
        u = lambda X: np.stack([X[:, 0] ** 2, 0 * X[:, 0], 0 * X[:, 0]], axis=1)
        ref_u = math.sqrt(1.0 / 5.0)
    p = lambda X: X[:, 0].copy()
    wl = _PolyWorkload(u, p)
    hy = StokesHierarchy((1, 1, 1), 1.0, 2, disc, coarse_level=2, workload=wl)
    lev = hy.lv[2]
    eu, ep = hy.error_norms(np.zeros(lev.size))
    assert eu == pytest.approx(ref_u, rel=1e-12)
    assert ep == pytest.approx(math.sqrt(1.0 / 12.0), rel=1e-12)
    uv = u(lev.vcoords())
    x = lev.join([uv[:, c] for c in range(3)], p(lev.pcoords()))
    eu0, ep0 = hy.error_norms(x)
    assert eu0 < 1e-13 and ep0 < 1e-13


def _dense_sgs_inverse(lev):
    """A_s^{-1} of the interior velocity block as a dense matrix: forward
    Gauss-Seidel (D + L)^{-1} in the stated order followed by the backward
    sweep, written as the two-step splitting form with triangular solves
    (not the oracle's phase loop)."""
    order = np.concatenate(lev.phases)
    A = lev.A[order][:, order].toarray()
    n = A.shape[0]
    low, up = np.tril(A), np.triu(A)
    F = np.linalg.solve(low, np.eye(n))                      # forward sweep from zero
    S = F + np.linalg.solve(up, np.eye(n) - A @ F)           # then the backward sweep
    return order, S


@pytest.mark.parametrize("disc,L", [("P1P1", 2), ("P2P1", 1)])
def test_omega_estimate_equals_dense_eigenvalue(disc, L):
    """The power iteration returns the largest eigenvalue of
    M_L^{-1}(C + B A_s^{-1} B^T), computed here densely with numpy.linalg.eigvals."""
    hy = StokesHierarchy((1, 1, 1), 1.0, L, disc, coarse_level=L, workload=Workload("curl"))
    lev = hy.lv[L]
    order, S = _dense_sgs_inverse(lev)
    B = [lev.B[c][:, order].toarray() for c in range(3)]
    T = lev.C.toarray() + sum(B[c] @ S @ B[c].T for c in range(3))
    T = T / lev.ML_hat[:, None]
    lam = np.max(np.abs(np.linalg.eigvals(T)))
    v0 = np.random.default_rng(0).uniform(-1, 1, lev.np)
    est = hy.estimate_omega_inv(v0, iters=400)
    assert est == pytest.approx(lam, rel=1e-6), (est, lam)


@pytest.mark.parametrize("disc,ahat", [("P1P1", "s"), ("P1P1", "f"), ("P2P1", "f")])
def test_uzawa_fixed_point_and_pressure_step(disc, ahat):
    """Eqs. uzawa-velocity / uzawa-pressure: the discrete solution (dense
    bordered solve) is a fixed point; and from (u*, p* + d) with a mean-zero
    pressure perturbation d, one iteration gives exactly
    u' = u* - A_hat^{-1} B^T d (dense splitting matrices) and
    p' = p* + d - S_hat^{-1}(B (u* - u') + C d), S_hat = omega^{-1} M_L."""
    L = 2 if disc == "P1P1" else 1
    hy = StokesHierarchy((1, 1, 1), 1.0, L, disc, coarse_level=L, workload=Workload("curl"))
    lev = hy.lv[L]
    b = hy.rhs[L]
    xs = lev.project_pressure(hy.coarse_solve(b))
    prm = Params(ahat=ahat, xi=1, omega_inv=0.7)
    x1 = lev.uzawa(xs, b, prm)
    assert np.linalg.norm(x1 - xs) <= 1e-11 * np.linalg.norm(xs)
    rng = np.random.default_rng(5)
    d = rng.uniform(-1, 1, lev.np)
    d -= np.dot(lev.ML, d) / lev.ML.sum()
    us, ps = lev.split(xs)
    x2 = lev.uzawa(lev.join(us, ps + d), b, prm)
    u2, p2 = lev.split(x2)
    order = np.concatenate(lev.phases)
    A = lev.A[order][:, order].toarray()
    if ahat == "f":
        Ainv = np.linalg.solve(np.tril(A), np.eye(A.shape[0]))
    else:
        _, Ainv = _dense_sgs_inverse(lev)
    Bd = [lev.B[c][:, order].toarray() for c in range(3)]
    du = []
    for c in range(3):
        ref = us[c].copy()
        ref[order] = us[c][order] - Ainv @ (Bd[c].T @ d)
        assert np.abs(u2[c] - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
        du.append(us[c] - u2[c])
    pref = ps + d - (sum(lev.B[c] @ du[c] for c in range(3)) + lev.C @ d) / (0.7 * lev.ML_hat)
    assert np.abs(p2 - pref).max() <= 1e-12 * max(1.0, np.abs(pref).max())
