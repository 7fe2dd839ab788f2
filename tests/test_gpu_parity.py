"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle on
the same seeded inputs.

Tolerances (FP64): 1e-12 relative per operator application and smoother
step, 1e-10 relative per V-cycle / FMG solve.  Boxes are chosen to span
several thread blocks and ragged tails (non-cubic boxes, odd extents).
"""
import numpy as np
import pytest
import torch

from gpu_helpers import OMEGA_INV, curl_workload, lib_problem, oracle_hierarchy, random_vector, rel

pytestmark = pytest.mark.gpu

APPLY_CASES = [
    ("P1P1", (1, 1, 1), 3, 0.0),
    ("P1P1", (2, 1, 3), 2, 0.0),
    ("P1P1", (1, 2, 1), 3, 1.7),
    ("P2P1", (1, 1, 1), 3, 0.0),
    ("P2P1", (2, 1, 1), 2, 0.0),
    ("P2P1", (1, 1, 2), 2, 1.1),
]


@pytest.mark.parametrize("disc,box,L,nu_a", APPLY_CASES)
def test_apply_parity(disc, box, L, nu_a):
    pb = lib_problem(box, L, disc, lc=1, nu_a=nu_a)
    hy = oracle_hierarchy(box, L, disc, lc=1, nu_a=nu_a)
    lev = hy.lv[L]
    x = random_vector(lev, 0)
    xd = pb.to_device(L, x)
    y = pb.new_vector(L)
    for op in ("FULL", "A", "BT", "B", "C"):
        pb.apply(L, op, xd, y)
        ref = lev.apply(x) if op == "FULL" else lev.apply_block(op, x)
        got = pb.to_host(L, y)
        if np.linalg.norm(ref) == 0:
            assert np.abs(got).max() == 0
        else:
            assert rel(got, ref) < 1e-12, (op, rel(got, ref))
    # mass matrix including Dirichlet rows, on a vector with boundary values
    xf = random_vector(lev, 1, zero_dirichlet=False)
    pb.apply(L, "MASS", pb.to_device(L, xf), y)
    assert rel(pb.to_host(L, y), lev.apply_block("MASS", xf)) < 1e-12


@pytest.mark.parametrize("disc,box,L,lc", [("P1P1", (1, 1, 1), 3, 0), ("P2P1", (1, 2, 1), 3, 1)])
def test_rhs_parity(disc, box, L, lc):
    wl = curl_workload() if box == (1, 1, 1) else __import__("hhg_inputs").Workload("modes", seed=3, box=box)
    pb = lib_problem(box, L, disc, lc=lc, workload=wl)
    hy = oracle_hierarchy(box, L, disc, lc=lc, workload=wl)
    for l in range(lc, L + 1):
        got = pb.to_host(l, pb.level_vector(l, "rhs"))
        assert rel(got, hy.rhs[l]) < 1e-12, (l, rel(got, hy.rhs[l]))
        gotW = pb.to_host(l, pb.level_vector(l, "W"))
        assert rel(gotW, hy.W[l]) < 1e-14 or np.linalg.norm(hy.W[l]) == 0


def test_set_rhs_levels_matches_per_level():
    """hhg_set_rhs_levels (every level queued, one synchronisation) assembles
    the same right-hand sides, bit for bit, as hhg_set_rhs level by level; an
    empty level range and a range with an invalid level or pointer are
    rejected without changing any level."""
    import ctypes as C
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    wl = Workload("modes", seed=5, box=(1, 2, 1))
    pb = lib_problem((1, 2, 1), 3, "P2P1", lc=1, workload=wl)
    ref = {l: pb.to_host(l, pb.level_vector(l, "rhs")) for l in (1, 2, 3)}
    fs, ws = [], []
    for l in (1, 2, 3):
        X = hhg.velocity_coords(pb.layout(l))
        fs.append(np.ascontiguousarray(wl.forcing(X).T.ravel()))
        ws.append(np.ascontiguousarray(wl.dirichlet(X).T.ravel()))
        pb.set_rhs(l, np.zeros_like(fs[-1]), np.zeros_like(ws[-1]))
    assert np.abs(pb.to_host(3, pb.level_vector(3, "rhs"))).max() == 0
    pb.set_rhs_levels(1, fs, ws)
    for l in (1, 2, 3):
        assert np.array_equal(pb.to_host(l, pb.level_vector(l, "rhs")), ref[l]), l
    dp = C.POINTER(C.c_double)
    assert hhg.load().hhg_set_rhs_levels(pb.h, 3, 2, (dp * 1)(), (dp * 1)()) == -1
    # a range that fails part-way (level 4 is beyond the hierarchy, or one
    # inner pointer is null) is rejected before anything is queued: no level
    # changes, although the earlier levels' data are valid
    zf = [np.zeros_like(f) for f in fs] + [np.zeros_like(fs[-1])]
    zw = [np.zeros_like(w) for w in ws] + [np.zeros_like(ws[-1])]
    fp = (dp * 4)(*[hhg._dp(a) for a in zf])
    wp = (dp * 4)(*[hhg._dp(a) for a in zw])
    assert hhg.load().hhg_set_rhs_levels(pb.h, 1, 4, fp, wp) == -1
    wp3 = (dp * 3)(*[hhg._dp(a) for a in zw[:3]])
    wp3[2] = dp()
    assert hhg.load().hhg_set_rhs_levels(pb.h, 1, 3, (dp * 3)(*[hhg._dp(a) for a in zf[:3]]), wp3) == -1
    for l in (1, 2, 3):
        assert np.array_equal(pb.to_host(l, pb.level_vector(l, "rhs")), ref[l]), l


@pytest.mark.parametrize("disc,nu_a", [("P1P1", 0.0), ("P2P1", 0.0), ("P1P1", 1.5)])
def test_residual_and_norms(disc, nu_a):
    box, L = (1, 1, 2), 2
    pb = lib_problem(box, L, disc, lc=1, nu_a=nu_a)
    hy = oracle_hierarchy(box, L, disc, lc=1, nu_a=nu_a)
    lev = hy.lv[L]
    x, b = random_vector(lev, 2), random_vector(lev, 3)
    r = pb.new_vector(L)
    nr = pb.residual(L, pb.to_device(L, x), pb.to_device(L, b), r, norms=True)
    ref = lev.residual(x, b)
    assert rel(pb.to_host(L, r), ref) < 1e-12
    assert np.allclose(nr, lev.norms(ref), rtol=1e-12)


@pytest.mark.parametrize("disc,ahat,xi,nu_a", [("P1P1", "s", 1, 0.0), ("P1P1", "f", 2, 1.2), ("P2P1", "f", 3, 0.0),
                                               ("P2P1", "s", 1, 0.0)])
def test_uzawa_parity(disc, ahat, xi, nu_a):
    from oracle.stokes import Params
    from paper_2010_13513_gb300.hhg import Params as LParams
    box, L = (2, 1, 1), 2
    pb = lib_problem(box, L, disc, lc=1, nu_a=nu_a)
    hy = oracle_hierarchy(box, L, disc, lc=1, nu_a=nu_a)
    lev = hy.lv[L]
    x, b = random_vector(lev, 4), random_vector(lev, 5)
    om = OMEGA_INV[disc]
    xd = pb.to_device(L, x)
    pb.smooth(L, LParams.make(ahat=ahat, xi=xi, omega_inv=om), 2, xd, pb.to_device(L, b))
    prm = Params(ahat=ahat, xi=xi, omega_inv=om)
    ref = lev.uzawa(lev.uzawa(x, b, prm), b, prm)
    assert rel(pb.to_host(L, xd), ref) < 1e-12


@pytest.mark.parametrize("disc,box,L,nu_a,ahat,xi", [("P2P1", (1, 1, 1), 3, 0.0, "f", 2),
                                                      ("P2P1", (2, 1, 1), 3, 1.1, "s", 1),
                                                      ("P1P1", (1, 2, 1), 4, 0.0, "s", 1)])
def test_gs_lanes_match_oracle(disc, box, L, nu_a, ahat, xi):
    """Per-phase Gauss-Seidel launches with 1, 2 and 4 lanes per site (terms
    split among the lanes, sums added by shuffles): two Uzawa iterations
    against the oracle in FP64, and FP32 against FP64 one lane per site.
    Vertex-colour planes of 27 to 153 sites leave partly filled warps."""
    from oracle.stokes import Params
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem(box, L, disc, lc=1, nu_a=nu_a, solve="mixed")
    hy = oracle_hierarchy(box, L, disc, lc=1, nu_a=nu_a)
    lev = hy.lv[L]
    x, b = random_vector(lev, 41), random_vector(lev, 42)
    om = OMEGA_INV[disc]
    lprm = hhg.Params.make(ahat=ahat, xi=xi, omega_inv=om)
    prm = Params(ahat=ahat, xi=xi, omega_inv=om)
    ref = lev.uzawa(lev.uzawa(x, b, prm), b, prm)
    pb.set_level_smoother(L, 0, prec=hhg.FP64)
    pb.set_level_smoother(L, 0, prec=hhg.FP32)
    for lanes, gs_threads in ((1, 128), (2, 64), (2, 256), (4, 64), (4, 128)):
        pb.set_launch_shape(L, 128, 2, gs_threads, 0, 1, lanes)
        assert pb.launch_shape(L)[5] == lanes
        xd = pb.to_device(L, x)
        pb.smooth(L, lprm, 2, xd, pb.to_device(L, b))
        assert rel(pb.to_host(L, xd), ref) < 1e-12, (lanes, gs_threads)
        x32 = pb.to_device(L, x, prec=hhg.FP32)
        pb.smooth(L, lprm, 2, x32, pb.to_device(L, b, prec=hhg.FP32))
        assert rel(pb.to_host(L, x32), ref) < 1e-4, (lanes, gs_threads)


@pytest.mark.parametrize("disc,L,nu_a,ahat,xi", [("P2P1", 2, 0.0, "s", 2), ("P2P1", 2, 1.3, "f", 1),
                                                  ("P1P1", 3, 0.0, "s", 1), ("P1P1", 3, 0.8, "f", 2)])
def test_resident_smoother_every_cta_count(disc, L, nu_a, ahat, xi):
    """The shared-memory-resident smoother on 1, 2, 4, 8 (and 16) CTAs, each
    owning a slab of k planes, gives the oracle's Uzawa iterates (FP64), and
    in FP32 the iterates of the per-phase launches up to rounding."""
    from oracle.stokes import Params
    from paper_2010_13513_gb300 import hhg
    box = (1, 1, 2)
    pb = lib_problem(box, L, disc, lc=1, nu_a=nu_a, solve="mixed")
    hy = oracle_hierarchy(box, L, disc, lc=1, nu_a=nu_a)
    lev = hy.lv[L]
    x, b = random_vector(lev, 14), random_vector(lev, 15)
    om = OMEGA_INV[disc]
    lprm = hhg.Params.make(ahat=ahat, xi=xi, omega_inv=om)
    prm = Params(ahat=ahat, xi=xi, omega_inv=om)
    ref = lev.uzawa(lev.uzawa(x, b, prm), b, prm)
    tried = []
    out32 = {}
    for ctas in (0, 1, 2, 4, 8, 16):
        try:
            pb.set_level_smoother(L, ctas, prec=hhg.FP64)
        except hhg.HHGError:
            continue
        assert pb.level_smoother(L, prec=hhg.FP64) == (ctas, 1024)
        xd = pb.to_device(L, x)
        pb.smooth(L, lprm, 2, xd, pb.to_device(L, b))
        assert rel(pb.to_host(L, xd), ref) < 1e-12, ctas
        tried.append(ctas)
        pb.set_level_smoother(L, ctas, prec=hhg.FP32)
        x32 = pb.to_device(L, x, prec=hhg.FP32)
        pb.smooth(L, lprm, 2, x32, pb.to_device(L, b, prec=hhg.FP32))
        out32[ctas] = pb.to_host(L, x32)
    assert {0, 1, 2, 4, 8} <= set(tried)
    if disc == "P1P1":
        assert 16 in tried                  # 17 k planes: the non-portable 16-CTA cluster
    for threads in (128, 256, 512):         # fewer threads per CTA: same iterates up to rounding
        pb.set_level_smoother(L, 2, threads, prec=hhg.FP64)
        xd = pb.to_device(L, x)
        pb.smooth(L, lprm, 2, xd, pb.to_device(L, b))
        assert rel(pb.to_host(L, xd), ref) < 1e-12, threads
    for ctas, v in out32.items():               # terms of a row summed in another order
        assert rel(v, out32[0]) < 1e-5, ctas
        assert rel(v, ref) < 1e-4


@pytest.mark.parametrize("disc,box,L,nu_a", [("P2P1", (4, 1, 1), 4, 0.0), ("P2P1", (4, 1, 1), 4, 1.1),
                                              ("P1P1", (4, 1, 2), 4, 0.0), ("P1P1", (4, 2, 1), 4, 0.9)])
def test_stream_rows_match_oracle(disc, box, L, nu_a):
    """The streaming row kernels (planes staged in shared memory, a quad of
    sites per thread, one or three passes) on levels with nx = 64 (the pitch
    of such levels is a multiple of four): the full operator and the B^T
    block against the oracle in FP64 (1e-12), the residual and the per-phase
    smoother's B^T and (B, -C) residual rows against the plain kernels (FP64
    1e-14, FP32 1e-6), for 64/128/256 threads per block of 4 sites per
    thread, or (FP32; FP64 keeps 4) 2 sites per thread (FP64 P2-P1 with 256
    threads exceeds the shared memory and falls back to the plain kernels);
    the planes of 17 or 33 rows of 68 positions end in partial tiles."""
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem(box, L, disc, lc=1, nu_a=nu_a, solve="mixed")
    hy = oracle_hierarchy(box, L, disc, lc=1, nu_a=nu_a)
    lev = hy.lv[L]
    assert pb.layout(L).sx % 4 == 0
    x, b = random_vector(lev, 21), random_vector(lev, 22)
    ref, ref_bt = lev.apply(x), lev.apply_block("BT", x)
    prm = hhg.Params.make(ahat="s", xi=1, omega_inv=OMEGA_INV[disc])
    pb.set_level_smoother(L, 0, prec=hhg.FP64)
    pb.set_level_smoother(L, 0, prec=hhg.FP32)
    out = {}
    for st, kc, v in ((0, 2, 1), (64, 3, 1), (128, 16, 2), (256, 5, 1), (128, 1, 1), (256, 4, 2), (64, 8, 2)):
        pb.set_launch_shape(L, 128, kc, 128, st, v)
        assert pb.launch_shape(L)[3] == st
        res = []
        for prec in (hhg.FP64, hhg.FP32):
            xd, bd = pb.to_device(L, x, prec=prec), pb.to_device(L, b, prec=prec)
            y, ybt, r = pb.new_vector(L, prec), pb.new_vector(L, prec), pb.new_vector(L, prec)
            pb.apply(L, "FULL", xd, y)
            pb.apply(L, "BT", xd, ybt)
            pb.residual(L, xd, bd, r)
            pb.smooth(L, prm, 1, xd, bd)
            res += [pb.to_host(L, v) for v in (y, ybt, r, xd)]
        assert rel(res[0], ref) < 1e-12, (st, kc, rel(res[0], ref))
        assert rel(res[1], ref_bt) < 1e-12, (st, kc, rel(res[1], ref_bt))
        assert rel(res[4], ref) < 1e-5
        out[(st, kc, v)] = res
    base = out[(0, 2, 1)]
    for key, res in out.items():
        for n, (a, c) in enumerate(zip(res, base)):
            assert rel(a, c) < (1e-14 if n < 4 else 1e-6), (key, n, rel(a, c))


@pytest.mark.parametrize("disc,box,L,nu_a", [("P2P1", (1, 1, 1), 4, 0.0), ("P2P1", (2, 1, 1), 3, 1.1),
                                              ("P1P1", (1, 2, 1), 4, 0.0), ("P1P1", (1, 1, 2), 3, 1.7)])
def test_row_sites_match_oracle(disc, box, L, nu_a):
    """Row kernels with 4 sites per thread (four runs of 32 positions of the
    padded plane per warp): the FP64 apply against the oracle, and apply,
    residual and the per-phase smoother's B^T and (B, -C) residual rows
    against one site per thread in FP64 and FP32.  The boxes give planes of
    97 to 625 positions: whole runs, a partial last warp, and warps with only
    the per-site tail."""
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem(box, L, disc, lc=1, nu_a=nu_a, solve="mixed")
    hy = oracle_hierarchy(box, L, disc, lc=1, nu_a=nu_a)
    lev = hy.lv[L]
    x, b = random_vector(lev, 31), random_vector(lev, 32)
    ref = lev.apply(x)
    prm = hhg.Params.make(ahat="s", xi=1, omega_inv=OMEGA_INV[disc])
    pb.set_level_smoother(L, 0, prec=hhg.FP64)
    pb.set_level_smoother(L, 0, prec=hhg.FP32)
    out = {}
    for sites, threads, kp in ((1, 128, 2), (4, 64, 4), (4, 256, 1), (4, 128, 3)):
        pb.set_launch_shape(L, threads, kp, 128, 0, sites)
        assert pb.launch_shape(L) == (threads, kp, 128, 0, sites, 1)
        res = []
        for prec in (hhg.FP64, hhg.FP32):
            xd, bd = pb.to_device(L, x, prec=prec), pb.to_device(L, b, prec=prec)
            y, r = pb.new_vector(L, prec), pb.new_vector(L, prec)
            pb.apply(L, "FULL", xd, y)
            pb.residual(L, xd, bd, r)
            pb.smooth(L, prm, 1, xd, bd)
            res += [pb.to_host(L, v) for v in (y, r, xd)]
        assert rel(res[0], ref) < 1e-12, (sites, rel(res[0], ref))
        assert rel(res[3], ref) < 1e-5
        out[(sites, threads, kp)] = res
    base = out[(1, 128, 2)]
    for key, res in out.items():
        for n, (a, c) in enumerate(zip(res, base)):
            assert rel(a, c) < (1e-14 if n < 3 else 1e-6), (key, n, rel(a, c))


def test_resident_smoother_rejects_what_does_not_fit():
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem((1, 1, 1), 3, "P2P1", lc=1)
    with pytest.raises(hhg.HHGError):
        pb.set_level_smoother(2, 8)          # 5 k planes on level 2
    with pytest.raises(hhg.HHGError):
        pb.set_level_smoother(3, -1)
    with pytest.raises(hhg.HHGError):
        pb.set_level_smoother(3, 17)
    with pytest.raises(hhg.HHGError):
        pb.set_level_smoother(3, 1, 100)     # not a multiple of 32
    pb.set_level_smoother(3, 0)
    assert pb.level_smoother(3)[0] == 0


@pytest.mark.parametrize("disc,box", [("P1P1", (2, 1, 1)), ("P2P1", (1, 1, 2)), ("P2P1", (1, 1, 1))])
def test_transfer_parity(disc, box):
    L = 2
    pb = lib_problem(box, L, disc, lc=1)
    hy = oracle_hierarchy(box, L, disc, lc=1)
    fine, coarse = hy.lv[2], hy.lv[1]
    xc = random_vector(coarse, 6)
    xf = random_vector(fine, 7)
    xfd = pb.to_device(2, xf)
    pb.prolongate_add(2, pb.to_device(1, xc), xfd)
    assert rel(pb.to_host(2, xfd), xf + hy.prolongate(2, xc)) < 1e-13
    rc = pb.new_vector(1)
    pb.restrict(2, pb.to_device(2, xf), rc)
    assert rel(pb.to_host(1, rc), hy.restrict(2, xf)) < 1e-13


@pytest.mark.parametrize("disc,lc", [("P1P1", 0), ("P1P1", 1), ("P2P1", 1)])
def test_coarse_solve_parity(disc, lc):
    box = (1, 1, 1)
    wl = curl_workload()
    pb = lib_problem(box, lc, disc, lc=lc, workload=wl)
    hy = oracle_hierarchy(box, lc, disc, lc=lc, workload=wl)
    b = hy.rhs[lc]
    x = pb.new_vector(lc)
    pb.coarse_solve(pb.to_device(lc, b), x)
    assert rel(pb.to_host(lc, x), hy.coarse_solve(b)) < 1e-11


@pytest.mark.parametrize("disc,L,lc,nu_a", [("P1P1", 3, 0, 0.0), ("P2P1", 3, 1, 0.0), ("P1P1", 3, 1, 2.0)])
def test_vcycle_parity(disc, L, lc, nu_a):
    from oracle.stokes import Params
    from paper_2010_13513_gb300.hhg import Params as LParams
    box = (1, 1, 1)
    wl = curl_workload(nu_a)
    pb = lib_problem(box, L, disc, lc=lc, nu_a=nu_a, workload=wl)
    hy = oracle_hierarchy(box, L, disc, lc=lc, nu_a=nu_a, workload=wl)
    om = OMEGA_INV[disc]
    s = dict(nu_pre=2, nu_post=1, nu_inc=1, kappa=1, ahat="f", xi=2, omega_inv=om)
    x = random_vector(hy.lv[L], 8)
    xd = pb.to_device(L, x)
    b = pb.level_vector(L, "rhs")
    # dirty the library's coarse work vectors first (a previous solve)
    pb.fmg_solve(LParams.make(**s), None, stats=False)
    pb.vcycle(L, LParams.make(**s), xd, b)
    ref = hy.vcycle(L, L, x, hy.rhs[L], Params(**s))
    assert rel(pb.to_host(L, xd), ref) < 1e-10


FMG_CASES = [
    # the P1-P1 PSPG workload on the 6-tetrahedron cube, level 4, V(3,3)
    ("P1P1", (1, 1, 1), 4, 0, 0.0, dict(nu_pre=3, nu_post=3, nu_inc=0, kappa=1, ahat="s", xi=1)),
    ("P2P1", (1, 1, 1), 3, 1, 0.0, dict(nu_pre=1, nu_post=3, nu_inc=2, kappa=1, ahat="f", xi=3)),
    ("P1P1", (2, 2, 2), 2, 0, 1.8, dict(nu_pre=2, nu_post=2, nu_inc=1, kappa=2, ahat="f", xi=1)),
]


@pytest.mark.parametrize("disc,box,L,lc,nu_a,s", FMG_CASES)
def test_fmg_parity(disc, box, L, lc, nu_a, s):
    from oracle.stokes import Params
    from paper_2010_13513_gb300.hhg import Params as LParams
    wl = curl_workload(nu_a)
    pb = lib_problem(box, L, disc, lc=lc, nu_a=nu_a, workload=wl)
    hy = oracle_hierarchy(box, L, disc, lc=lc, nu_a=nu_a, workload=wl)
    om = OMEGA_INV[disc]
    x = pb.new_vector(L)
    st = pb.fmg_solve(LParams.make(**s, omega_inv=om), x)
    ref = hy.fmg(Params(**s, omega_inv=om))
    got = pb.to_host(L, x)
    assert rel(got, ref) < 1e-10, rel(got, ref)
    lev = hy.lv[L]
    assert np.allclose([st.res_u, st.res_p], lev.norms(lev.residual(ref, hy.rhs[L])), rtol=1e-6)
    assert st.kernel_launches > 0


def test_omega_estimate_parity():
    box, L = (1, 1, 1), 3
    pb = lib_problem(box, L, "P1P1", lc=1)
    hy = oracle_hierarchy(box, L, "P1P1", lc=1)
    v0 = np.random.default_rng(0).uniform(-1, 1, hy.lv[L].np)
    got = pb.estimate_omega(L, v0, iters=30)
    ref = hy.estimate_omega_inv(v0, iters=30)
    assert abs(got / ref - 1) < 1e-10


@pytest.mark.parametrize("disc,L,lc", [("P1P1", 3, 0), ("P2P1", 2, 1)])
def test_error_norms_parity(disc, L, lc):
    from paper_2010_13513_gb300.hhg import pressure_coords, velocity_coords
    from oracle.stokes import StokesLevel
    box = (1, 1, 1)
    wl = curl_workload()
    pb = lib_problem(box, L, disc, lc=lc, workload=wl, error_level=True)
    hy = oracle_hierarchy(box, L, disc, lc=lc, workload=wl)
    x = random_vector(hy.lv[L], 9) * 0.01
    info = pb.layout(L + 1)
    ue = wl.exact_velocity(velocity_coords(info)).T.ravel()
    pe = wl.exact_pressure(pressure_coords(info))
    got = pb.error_norms(L, pb.to_device(L, x), ue, pe)
    ref = hy.error_norms(x)
    assert np.allclose(got, ref, rtol=1e-11)


def test_mixed_precision_close_to_fp64_oracle():
    """FP32 V-cycles inside FP64 refinement: reported error against the FP64
    oracle (no parity claim); it must be far below the discretisation error."""
    from oracle.stokes import Params
    from paper_2010_13513_gb300.hhg import Params as LParams
    box, L, lc = (1, 1, 1), 4, 0
    wl = curl_workload()
    s = dict(nu_pre=3, nu_post=3, nu_inc=0, kappa=1, ahat="s", xi=1, omega_inv=0.5)
    pb = lib_problem(box, L, "P1P1", lc=lc, solve="mixed", workload=wl)
    hy = oracle_hierarchy(box, L, "P1P1", lc=lc, workload=wl)
    x = pb.new_vector(L)
    pb.fmg_solve(LParams.make(**s), x)
    ref = hy.fmg(Params(**s))
    err = rel(pb.to_host(L, x), ref)
    print(f"mixed-precision FMG vs FP64 oracle: relative difference {err:.3e}")
    assert err < 1e-5


def _abs_row_sums(lev, x):
    """s_i = sum_j |a_ij x_j| of the oracle's operator rows."""
    u, p = lev.split(np.abs(x))
    su = [abs(lev.A) @ u[c] + abs(lev.B[c]).T @ p for c in range(3)]
    sp = sum(abs(lev.B[c]) @ u[c] for c in range(3)) + abs(lev.C) @ p
    return lev.join(su, sp)


@pytest.mark.parametrize("disc,box,L,H,nu_a", [("P2P1", (1, 1, 1), 3, 1.0, 0.0), ("P1P1", (2, 2, 2), 3, 0.5, 0.0),
                                               ("P1P1", (1, 2, 1), 4, 1.0, 0.0), ("P1P1", (2, 2, 2), 3, 0.5, 1.7),
                                               ("P2P1", (1, 1, 1), 3, 1.0, 1.3)])
def test_refinement_residual_double_float(disc, box, L, H, nu_a):
    """The mixed solve's refinement defect r = fl32(b - calA x)
    (hhg_refinement_residual) in double-float arithmetic and in FP64, against
    the oracle's FP64 residual, entrywise:
        |r_i - r_i^oracle| <= 2^-24 |r_i^oracle| + 2^-32 (s_i + |b_i|),
    s_i = sum_j |a_ij x_j|.  b = calA x + 1e-6 noise, so each row cancels to
    about 1e-6 s_i: a row summed in plain FP32 (error ~ n 2^-24 s_i) misses
    the bound by orders of magnitude, a dropped low part (2^-24 s_i) too.
    P1-P1 boxes exercise the clipped C terms of the boundary pressure rows;
    the 1 x 2 x 1 box at level 4 leaves a partly filled last warp; nu_a != 0
    (nu = exp(nu_a z)) the segments scaled by the rows' exp(+-nu_a h k)."""
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem(box, L, disc, lc=1, solve="mixed", H=H, nu_a=nu_a)
    hy = oracle_hierarchy(box, L, disc, lc=1, H=H, nu_a=nu_a)
    lev = hy.lv[L]
    x = random_vector(lev, 21)
    b = lev.apply(x) + 1e-6 * random_vector(lev, 22)
    ref = lev.residual(x, b)
    bound = 2.0 ** -24 * np.abs(ref) + 2.0 ** -32 * (_abs_row_sums(lev, x) + np.abs(b))
    assert pb.refinement_residual_kind() == "df32"
    xd, bd = pb.to_device(L, x), pb.to_device(L, b)
    for kind in ("df32", "fp64"):
        pb.set_refinement_residual(kind)
        assert pb.refinement_residual_kind() == kind
        r = pb.new_vector(L, prec=hhg.FP32)
        pb.refinement_residual(L, xd, bd, r)
        err = np.abs(pb.to_host(L, r) - ref)
        assert np.all(err <= bound), (kind, float((err / bound).max()))
    # plain FP32 rows on the same input miss the bound (the bound is sharp enough to tell)
    r32 = pb.new_vector(L, prec=hhg.FP32)
    pb.residual(L, pb.to_device(L, x, prec=hhg.FP32), pb.to_device(L, b, prec=hhg.FP32), r32)
    assert np.any(np.abs(pb.to_host(L, r32) - ref) > bound)


@pytest.mark.parametrize("disc,box,L,lc", [("P2P1", (1, 1, 1), 4, 2), ("P1P1", (1, 1, 1), 4, 0)])
def test_mixed_fmg_refinement_kinds_agree(disc, box, L, lc):
    """The mixed-precision FMG with the double-float refinement residual (the
    default) and with the FP64 one: both within 1e-5 of the FP64 oracle's FMG
    and within 1e-6 of each other.  The two defects differ by ~2^-40 of the
    row sums before their rounding to FP32, which then differs in the last
    bit for some entries; the FP32 V-cycles carry that into corrections that
    differ at FP32 rounding (~1e-7 relative), not at the defects' 2^-40."""
    from oracle.stokes import Params
    from paper_2010_13513_gb300.hhg import Params as LParams
    wl = curl_workload()
    s = dict(nu_pre=3, nu_post=3, nu_inc=0, kappa=1, ahat="s", xi=1, omega_inv=OMEGA_INV[disc])
    pb = lib_problem(box, L, disc, lc=lc, solve="mixed", workload=wl)
    ref = oracle_hierarchy(box, L, disc, lc=lc, workload=wl).fmg(Params(**s))
    sols = {}
    for kind in ("df32", "fp64"):
        pb.set_refinement_residual(kind)
        x = pb.new_vector(L)
        pb.fmg_solve(LParams.make(**s), x)
        sols[kind] = pb.to_host(L, x)
        assert rel(sols[kind], ref) < 1e-5, kind
    assert rel(sols["df32"], sols["fp64"]) < 1e-6


def test_fp32_kernels_track_fp64():
    """FP32 apply of the same operator: relative difference at FP32 rounding."""
    box, L = (1, 1, 1), 3
    pb = lib_problem(box, L, "P2P1", lc=1, solve="mixed")
    hy = oracle_hierarchy(box, L, "P2P1", lc=1)
    lev = hy.lv[L]
    x = random_vector(lev, 10)
    y = pb.new_vector(L, prec=1)
    pb.apply(L, "FULL", pb.to_device(L, x, prec=1), y)
    assert rel(pb.to_host(L, y), lev.apply(x)) < 1e-5


def test_invalid_arguments_raise():
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem((1, 1, 1), 2, "P1P1", lc=0)
    with pytest.raises(hhg.HHGError):
        pb.apply(7, "FULL", pb.new_vector(2), pb.new_vector(2))
    with pytest.raises(hhg.HHGError):
        pb.fmg_solve(hhg.Params.make())             # no rhs set


def test_fmg_graph_replay_matches_direct_launches():
    """The CUDA-graph replay of a whole FMG solve issues the same kernels as
    the direct launches: results are bitwise equal, repeatedly."""
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pb = lib_problem((1, 1, 1), 3, "P2P1", lc=1, solve="mixed", workload=curl_workload())
    assert pb.stream == stream
    prm = hhg.Params.make(1, 3, 2, 1, "f", 3, 0.3)
    xg = pb.new_vector(3)
    st1 = pb.fmg_solve(prm, xg)                  # records and replays the graph
    st2 = pb.fmg_solve(prm, xg)                  # replays the cached graph
    pb.set_graph_mode(False)
    xd = pb.new_vector(3)
    st3 = pb.fmg_solve(prm, xd)
    stream.synchronize()
    assert torch.equal(xg, xd)
    assert st1.kernel_launches == st2.kernel_launches == st3.kernel_launches
    assert st1.res_u == st3.res_u and st1.res_p == st3.res_p


@pytest.mark.parametrize("disc,L,lc,solve,ahat", [("P2P1", 4, 1, "mixed", "f"), ("P1P1", 4, 0, "fp64", "s"),
                                                  ("P1P1", 3, 1, "mixed", "s")])
def test_cluster_smoother_matches_per_phase_launches(disc, L, lc, solve, ahat):
    """Small levels run all smoother phases in one thread-block-cluster launch;
    the FMG result equals that of one launch per phase up to the rounding of
    the V-cycle precision (the resident kernel adds the terms of a row in
    another order)."""
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem((1, 1, 1), L, disc, lc=lc, solve=solve, workload=curl_workload())
    prm = hhg.Params.make(1, 3, 2, 1, ahat, 2, OMEGA_INV[disc])
    assert any(pb.level_smoother(l)[0] > 0 for l in range(lc, L + 1))
    x1 = pb.new_vector(L)
    pb.fmg_solve(prm, x1, stats=False)
    pb.set_small_level_mode(False)
    x2 = pb.new_vector(L)
    pb.fmg_solve(prm, x2, stats=False)
    torch.cuda.synchronize()
    assert rel(x1.cpu().numpy(), x2.cpu().numpy()) < (1e-13 if solve == "fp64" else 1e-5)


def test_batch_graph_matches_individual_solves():
    """A batch of uneven problems (P1-P1 / P2-P1, different boxes, levels and
    precisions) solved by one graph gives exactly the individual FMG
    results."""
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    specs = [("P1P1", (1, 1, 1), 3, 0, "fp64"), ("P2P1", (2, 1, 1), 3, 1, "mixed"),
             ("P1P1", (1, 2, 2), 2, 0, "mixed"), ("P2P1", (1, 1, 1), 2, 1, "fp64")]
    pbs, prms, refs = [], [], []
    with torch.cuda.stream(stream):
        for i, (disc, box, L, lc, solve) in enumerate(specs):
            wl = Workload("modes", seed=100 + i, box=box, H=1.0 / max(box))
            pbs.append(lib_problem(box, L, disc, lc=lc, solve=solve, workload=wl))
            prms.append(hhg.Params.make(1, 2, 1, 1, "f", 2, OMEGA_INV[disc]))
        batch = hhg.Batch(pbs)            # gives the problems common launch shapes
        for pb, prm in zip(pbs, prms):
            x = pb.new_vector(pb.L)
            pb.fmg_solve(prm, x, stats=False)
            refs.append(x.clone())
        for rep in range(2):
            k = batch.fmg_solve(prms, stream)
        stream.synchronize()
    # four different sequence structures: nothing to merge (each problem is
    # its own cohort, and its zeroing copies become kernels)
    launches, own = batch.launch_counts()
    assert launches == k and k >= own > 0
    for pb, ref in zip(pbs, refs):
        got = pb.level_vector(pb.L, "x")
        assert torch.equal(got, ref)


def test_batch_merges_aligned_problems():
    """Problems whose kernel sequences align (same discretisation, level and
    parameters; boxes of different shape) share their launches, and every
    problem still gets exactly its individual FMG result (the resident cluster
    smoother, the row and Gauss-Seidel kernels, transfers, reductions and the
    coarse solve all run as merged work-item lists)."""
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    specs = [("P2P1", (1, 1, 1)), ("P2P1", (2, 1, 1)), ("P2P1", (1, 2, 1)), ("P2P1", (1, 1, 2)),
             ("P1P1", (1, 1, 1)), ("P1P1", (2, 2, 1)), ("P1P1", (1, 2, 2))]
    pbs, prms, refs = [], [], []
    own_each = []
    with torch.cuda.stream(stream):
        for i, (disc, box) in enumerate(specs):
            wl = Workload("modes", seed=200 + i, box=box, H=1.0 / max(box))
            lc = 1 if disc == "P2P1" else 0
            pbs.append(lib_problem(box, 4, disc, lc=lc, solve="mixed", workload=wl))
            prms.append(hhg.Params.make(1, 2, 1, 1, "f", 2, OMEGA_INV[disc]))
        batch = hhg.Batch(pbs)            # gives the problems common launch shapes
        for pb, prm in zip(pbs, prms):
            x = pb.new_vector(4)
            st = pb.fmg_solve(prm, x)
            own_each.append(st.kernel_launches)
            refs.append(x.clone())
        counts = {}
        for grouping in (1, 0, 2):
            batch.set_grouping(grouping)
            for pb in pbs:
                pb.level_vector(pb.L, "x").zero_()
            batch.fmg_solve(prms, stream)
            batch.fmg_solve(prms, stream)
            stream.synchronize()
            counts[grouping] = batch.launch_counts()
            for pb, ref in zip(pbs, refs):
                assert torch.equal(pb.level_vector(pb.L, "x"), ref), grouping
    # grouping 1 (cohorts by structure): seven sequences in less than half the
    # launches (problems whose smoother runs on clusters of different sizes
    # cannot share those launches); grouping 0 (identical sequences only)
    # merges less; grouping 2 merges nothing
    assert all(own == sum(own_each) for _, own in counts.values())
    assert counts[1][0] < sum(own_each) / 2, (counts, own_each)
    assert counts[1][0] <= counts[0][0] <= counts[2][0] + 50, counts


def test_batch_variable_viscosity_matches_individual_solves():
    """Mixed-precision problems with nu = exp(a z) in one batch (the
    double-float defect's variable-viscosity kernels as merged work items):
    every problem gets exactly its individual FMG result, merged and not."""
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    specs = [("P1P1", (1, 1, 1), 0.9), ("P1P1", (2, 1, 1), 0.9), ("P2P1", (1, 1, 1), 1.4)]
    pbs, prms, refs = [], [], []
    with torch.cuda.stream(stream):
        for i, (disc, box, nu_a) in enumerate(specs):
            wl = Workload("modes", seed=300 + i, box=box, H=1.0 / max(box))
            pbs.append(lib_problem(box, 3, disc, lc=1, solve="mixed", nu_a=nu_a, workload=wl))
            prms.append(hhg.Params.make(1, 2, 1, 1, "f", 2, OMEGA_INV[disc]))
        batch = hhg.Batch(pbs)
        for pb, prm in zip(pbs, prms):
            assert pb.refinement_residual_kind() == "df32"
            x = pb.new_vector(3)
            pb.fmg_solve(prm, x, stats=False)
            refs.append(x.clone())
        for grouping in (1, 2):
            batch.set_grouping(grouping)
            for pb in pbs:
                pb.level_vector(pb.L, "x").zero_()
            batch.fmg_solve(prms, stream)
            stream.synchronize()
            for pb, ref in zip(pbs, refs):
                assert torch.equal(pb.level_vector(pb.L, "x"), ref), grouping


def test_autotune_keeps_results():
    from paper_2010_13513_gb300 import hhg
    pb = lib_problem((1, 1, 1), 4, "P2P1", lc=1, solve="mixed", workload=curl_workload())
    prm = hhg.Params.make(1, 3, 2, 1, "f", 3, 0.3)
    x1 = pb.new_vector(4)
    pb.fmg_solve(prm, x1, stats=False)
    shapes = pb.autotune(reps=2)
    assert set(shapes) == {1, 2, 3, 4}
    for t, kp, gs, rc, rt, tile, sites, lanes, lanes_v, btt, btk, bts, bct, bck, bcs, gsv in shapes.values():
        assert t in (64, 128, 256) and kp in (1, 2, 4, 8, 16) and gs in (64, 128, 256)
        assert rc in (0, 1, 2, 4, 8, 16) and rt in (256, 512, 1024) and tile in (0, 64, 128, 256) and sites in (1, 4)
        assert lanes in (1, 2, 4) and lanes_v in (1, 2, 4)
        assert btt in (64, 128, 256) and bct in (64, 128, 256) and btk in (1, 2, 4) and bck in (1, 2, 4)
        assert bts in (1, 4) and bcs in (1, 4) and gsv in (64, 128, 256)
    x2 = pb.new_vector(4)
    pb.fmg_solve(prm, x2, stats=False)
    torch.cuda.synchronize()
    # launch shapes do not change the arithmetic; the resident smoother's CTA
    # count changes the order of the FP32 partial sums of a row
    assert rel(x1.cpu().numpy(), x2.cpu().numpy()) < 1e-5


@pytest.mark.parametrize("graphs", [True, False])
def test_fmg_solve_host_matches_separate_calls(graphs):
    """hhg_fmg_solve_host (right-hand sides of every level from host nodal
    data, the finest one assembled on a second stream beside the FMG stages
    below it, the FMG, the solution to the host) gives exactly the result of
    hhg_set_rhs_levels + hhg_fmg_solve + hhg_vector_to_host, on repeated
    calls (the second replays the split graphs) and without graphs."""
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pb = lib_problem((1, 1, 1), 4, "P2P1", lc=1, solve="mixed")
        pb.set_graph_mode(graphs)
        wl = Workload("paper")
        f, w = [], []
        for l in range(1, 5):
            X = hhg.velocity_coords(pb.layout(l))
            f.append(torch.from_numpy(np.ascontiguousarray(wl.forcing(X).T.ravel())).pin_memory())
            w.append(torch.from_numpy(np.ascontiguousarray(wl.dirichlet(X).T.ravel())).pin_memory())
        prm = hhg.Params.make(1, 3, 1, 1, "f", 3, OMEGA_INV["P2P1"])
        pb.set_rhs_levels(1, f, w)
        x = pb.new_vector(4)
        st_ref = pb.fmg_solve(prm, x)
        ref = torch.from_numpy(np.array(pb.to_host(4, x)))
        out = torch.empty(pb.layout(4).n_dofs, dtype=torch.float64).pin_memory()
        for _ in range(3):
            out.zero_()
            st = pb.fmg_solve_host(prm, f, w, out=out)
            assert torch.equal(out, ref)
            assert st.res_u == st_ref.res_u and st.res_p == st_ref.res_p
            assert st.wu_counted == pytest.approx(st_ref.wu_counted, rel=1e-12)
