"""Plain FP64 reference of the matrix-free FMG Stokes solver (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Slow and direct: every
operator is a globally assembled sparse matrix built from exact element
matrices (oracle/fe.py), every solver step follows the paper's equations in
order.  It shares no code with the CUDA library.

Discrete system (Sec. 2, Eq. stokes-discrete):
    [A  B^T] [u]   [f]
    [B  -C ] [p] = [g],   A = diag(A, A, A)
with Dirichlet velocity nodes eliminated by lifting (Sec. 2, right-hand side
below Eq. stokes-discrete): the unknown vector holds interior velocity values
(boundary entries are kept as zeros) and all pressure values, and
    f_i = (M f_h)_i - sum_{j on boundary} a_ij w_j          (interior i)
    g_k = - sum_{j on boundary} b_kj w_j  [+ PSPG load, P1-P1]
where f_h is the nodal interpolant of f in the velocity space and M the
velocity mass matrix.  g is then projected onto the range of the operator
(sum_k g_k = 0), the only component a pure-Dirichlet problem can fit.

Vectors are flat numpy arrays [u_1, u_2, u_3, p]; velocity blocks span all
velocity nodes of the level (P1 lattice for P1-P1, doubled lattice for
P2-P1), the pressure block all P1 lattice nodes.

Smoother (Sec. 3.2, Eq. uzawa-iteration/-velocity/-pressure):
    u-step: f' = f - B^T p_k, then xi Gauss-Seidel sweeps (A_f: forward,
            A_s: forward + backward) on A u = f'
    p-step: p_{k+1} = p_k - S_hat^{-1} (g - B u_{k+1} + C p_k)
with S_hat = omega^{-1} M_L (lumped P1 pressure mass; with a variable
viscosity the lumped mass of 1/nu).  This is the positive, well-defined
reading of Sec. 3.2: omega^{-1} diag(-C) would be negative for P1-P1 and zero
for P2-P1 (C = 0), while the eigenproblem that defines omega^{-1} is
normalised by M_L.  Gauss-Seidel uses the multicolour order shared with the GPU: vertex
DoFs in 4 colours c = (i + j + k) mod 4, then (P2 only) the seven edge groups
x, y, z, xy, xz, yz, xyz, each of which has no coupling inside the group.

Multigrid (Algorithm 1): variable V-cycle with nu + (l_fine - l) nu_inc
sweeps, FMG with kappa cycles per level, direct coarse solve of the system
bordered by the pressure mean constraint.  Transfers (Sec. 3.3): nodal
interpolation (linear P1, quadratic P2), restriction = transpose.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fe
from .mesh import Lattice, PERMS

EDGE_GROUP_ORDER = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1), (0, 1, 1), (1, 1, 1)]


@dataclass
class Params:
    """The FMG parameter tuple s = (nu_pre, nu_post, nu_inc, kappa, A_hat, xi)
    of Algorithm 1 / Sec. 5.1, plus the pressure relaxation omega^{-1}."""
    nu_pre: int = 3
    nu_post: int = 3
    nu_inc: int = 0
    kappa: int = 1
    ahat: str = "s"       # "f" forward GS, "s" symmetric GS
    xi: int = 1
    omega_inv: float = 0.5


# =====================================================================
# one level of the hierarchy
# =====================================================================
class StokesLevel:
    def __init__(self, box, H, level, disc, nu_a=0.0, pspg_rhs=True):
        self.lat = lat = Lattice(box, H, level)
        self.disc = disc
        self.order_v = 1 if disc == "P1P1" else 2
        self.nu_a = float(nu_a)
        self.level = level
        self.np = lat.p1_count()
        self.nv = lat.p1_count() if self.order_v == 1 else lat.p2_count()

        tets, cls = lat.tets()
        # velocity and pressure DoF indices of each micro tetrahedron
        pdofs = lat.p1_index(tets)                                   # (nt, 4)
        if self.order_v == 1:
            vdofs = pdofs
        else:
            vpos = [2 * tets[:, a] for a in range(4)] + [tets[:, a] + tets[:, b] for a, b in fe.EDGES]
            vdofs = np.stack([lat.p2_index(v) for v in vpos], axis=1)  # (nt, 10)
        self.tet_vdofs, self.tet_pdofs = vdofs, pdofs

        # per-tet coefficient nu_T at the centroid (1 for constant viscosity)
        cent = tets.mean(axis=1) * lat.h
        nuT = np.exp(self.nu_a * cent[:, 2]) if self.nu_a != 0.0 else np.ones(tets.shape[0])

        nv, npp = self.nv, self.np
        A = _Assembler(nv, nv)
        Mv = _Assembler(nv, nv)
        Bd = [_Assembler(npp, nv) for _ in range(3)]
        Ld = [_Assembler(npp, nv) for _ in range(3)]
        C = _Assembler(npp, npp)
        Mp = _Assembler(npp, npp)
        MLnu = np.zeros(npp)
        for s in range(6):
            sel = np.nonzero(cls == s)[0]
            if sel.size == 0:
                continue
            X = tets[sel[0]].astype(np.float64) * lat.h
            X = X - X[0]                                   # geometry is translation invariant
            vd, pd, w = vdofs[sel], pdofs[sel], nuT[sel]
            A.add(vd, vd, fe.stiffness(X, self.order_v), w)
            Mv.add(vd, vd, fe.mass(X, self.order_v), None)
            D = fe.divergence(X, self.order_v)
            for d in range(3):
                Bd[d].add(pd, vd, D[d], None)
            if disc == "P1P1":
                C.add(pd, pd, fe.pspg(X), 1.0 / w)
                if pspg_rhs:
                    Ld_e = fe.pspg_load(X, self.order_v)
                    for d in range(3):
                        Ld[d].add(pd, vd, Ld_e[d], 1.0 / w)
            Mp.add(pd, pd, fe.mass(X, 1), None)
            vol, _ = fe.tet_geometry(X)
            np.add.at(MLnu, pd.ravel(), np.repeat(vol / 4.0 / w, 4))
        self.A = A.tocsr()
        self.Mv = Mv.tocsr()
        self.B = [b.tocsr() for b in Bd]
        self.L = [l.tocsr() for l in Ld]
        self.C = C.tocsr()
        self.Mp = self.Mp_full = Mp.tocsr()
        self.ML = np.asarray(self.Mp.sum(axis=1)).ravel()       # lumped P1 mass
        self.ML_hat = MLnu                                       # lumped mass of 1/nu

        bnd = lat.boundary_mask_p1() if self.order_v == 1 else lat.boundary_mask_p2()
        self.vbnd = bnd
        self.vint = ~bnd
        self.Adiag = self.A.diagonal()
        self.phases = self._gs_phases()
        self.gs_order = "multicolour"
        self._lex = None

    # ---------------------------------------------------------------- layout
    @property
    def size(self):
        return 3 * self.nv + self.np

    def split(self, x):
        nv = self.nv
        return [x[c * nv:(c + 1) * nv] for c in range(3)], x[3 * nv:]

    def join(self, u, p):
        return np.concatenate([u[0], u[1], u[2], p])

    def vcoords(self):
        return self.lat.p1_coords() if self.order_v == 1 else self.lat.p2_coords()

    def pcoords(self):
        return self.lat.p1_coords()

    # -------------------------------------------------------- GS colouring
    def _gs_phases(self):
        """Index sets of interior velocity DoFs, in forward GS order."""
        phases = []
        if self.order_v == 1:
            ijk = self.lat.p1_int_coords()
            col = ijk.sum(axis=1) % 4
            for c in range(4):
                phases.append(np.nonzero(self.vint & (col == c))[0])
            return phases
        IJK = self.lat.p2_int_coords()
        par = IJK % 2
        vert = np.all(par == 0, axis=1)
        col = (IJK // 2).sum(axis=1) % 4
        for c in range(4):
            phases.append(np.nonzero(self.vint & vert & (col == c))[0])
        for o in EDGE_GROUP_ORDER:
            g = np.all(par == np.array(o)[None, :], axis=1)
            phases.append(np.nonzero(self.vint & g)[0])
        return phases

    def set_gs_order(self, order):
        """'multicolour' (the order above, shared with the GPU) or 'paper':
        the order of the paper's Gauss-Seidel kernels (Sec. 5.2: one kernel
        per DoF group) -- the interior vertex DoFs one after another in
        lexicographic order (i fastest, then j, then k), then (P2) each edge
        group at once as above.  Backward = exact reverse."""
        if order not in ("multicolour", "paper"):
            raise ValueError(order)
        self.gs_order = order
        if order == "paper" and self._lex is None:
            V = np.sort(np.concatenate(self.phases[:4]))        # interior vertex DoFs, natural order
            AVV = self.A[V][:, V].tocsr()
            self._lex = (V, self.A[V].tocsr(), sp.tril(AVV, format="csr"), sp.triu(AVV, format="csr"))

    def _gs_vertices_lex(self, u, rhs, backward):
        """The vertex group, DoF by DoF in lexicographic order (reverse order
        for backward): u_V solves (D + L) u_V = rhs_V - (A u)_V + (D + L) u_V
        with the other DoFs fixed, L (or U) the strictly lower (upper)
        triangle of A restricted to V in that order -- each DoF's update sees
        the new values of the DoFs before it."""
        V, AV, low, up = self._lex
        T = up if backward else low
        r = rhs[V] - AV @ u + T @ u[V]
        u[V] = spla.spsolve_triangular(T, r, lower=not backward)

    # ------------------------------------------------------------ operators
    def apply(self, x):
        """y = calA x (Eq. stokes-discrete); Dirichlet velocity rows are 0."""
        u, p = self.split(x)
        yu = [np.where(self.vint, self.A @ u[c] + self.B[c].T @ p, 0.0) for c in range(3)]
        yp = sum(self.B[c] @ u[c] for c in range(3)) - self.C @ p
        return self.join(yu, yp)

    def apply_block(self, op, x):
        """Single blocks: 'A' (vector Laplacian), 'BT', 'B', 'C', 'MASS'."""
        u, p = self.split(x)
        z = np.zeros(self.nv)
        if op == "A":
            return self.join([np.where(self.vint, self.A @ u[c], 0.0) for c in range(3)], np.zeros(self.np))
        if op == "BT":
            return self.join([np.where(self.vint, self.B[c].T @ p, 0.0) for c in range(3)], np.zeros(self.np))
        if op == "B":
            return self.join([z, z, z], sum(self.B[c] @ u[c] for c in range(3)))
        if op == "C":
            return self.join([z, z, z], self.C @ p)
        if op == "MASS":
            return self.join([self.Mv @ u[c] for c in range(3)], self.Mp @ p)
        raise ValueError(op)

    def residual(self, x, b):
        return b - self.apply(x)

    def norms(self, r):
        u, p = self.split(r)
        return float(np.sqrt(sum(np.dot(uc, uc) for uc in u))), float(np.linalg.norm(p))

    # ------------------------------------------------------------ smoother
    def gs_sweep(self, u, rhs, backward=False):
        """One Gauss-Seidel sweep on A u = rhs (in place), in the level's
        order (multicolour, or the paper's: see set_gs_order)."""
        A, d = self.A, self.Adiag
        if self.gs_order == "paper":
            edges = self.phases[4:]
            if not backward:
                self._gs_vertices_lex(u, rhs, False)
            for S in (edges[::-1] if backward else edges):
                if S.size:
                    u[S] = (rhs[S] - A[S] @ u + d[S] * u[S]) / d[S]
            if backward:
                self._gs_vertices_lex(u, rhs, True)
            return
        order = self.phases[::-1] if backward else self.phases
        for S in order:
            if S.size == 0:
                continue
            u[S] = (rhs[S] - A[S] @ u + d[S] * u[S]) / d[S]

    def uzawa(self, x, b, prm: Params):
        """One inexact Uzawa iteration, Eq. uzawa-velocity then Eq. uzawa-pressure."""
        u, p = self.split(x.copy())
        f, g = self.split(b)
        fprime = [np.where(self.vint, f[c] - self.B[c].T @ p, 0.0) for c in range(3)]
        for _ in range(prm.xi):
            for c in range(3):
                self.gs_sweep(u[c], fprime[c], backward=False)
                if prm.ahat == "s":
                    self.gs_sweep(u[c], fprime[c], backward=True)
        rp = g - sum(self.B[c] @ u[c] for c in range(3)) + self.C @ p
        p = p - rp / (prm.omega_inv * self.ML_hat)
        return self.join(u, p)

    def project_pressure(self, x):
        """Remove the constant pressure mode: int p_h = 1^T M_L p = 0."""
        u, p = self.split(x)
        p = p - np.dot(self.ML, p) / self.ML.sum()
        return self.join(u, p)

    # ----------------------------------------------------------------- rhs
    def assemble_rhs(self, workload):
        """b = [f; g] from the forcing f and Dirichlet data w (nodal interpolants)."""
        Xv = self.vcoords()
        fn = workload.forcing(Xv)                 # (nv, 3)
        wn = workload.dirichlet(Xv) * self.vbnd[:, None]
        f = [np.where(self.vint, self.Mv @ fn[:, c] - self.A @ wn[:, c], 0.0) for c in range(3)]
        g = -sum(self.B[c] @ wn[:, c] for c in range(3))
        if self.disc == "P1P1":
            g = g + sum(self.L[c] @ fn[:, c] for c in range(3))
        g = g - g.mean()
        W = self.join([wn[:, c] for c in range(3)], np.zeros(self.np))
        return self.join(f, g), W


class _Assembler:
    """COO accumulation of element contributions: M = sum_T P_T^T K_T P_T."""

    def __init__(self, nr, nc):
        self.nr, self.nc = nr, nc
        self.rows, self.cols, self.vals = [], [], []

    def add(self, rdofs, cdofs, Ke, scale):
        nt, nr = rdofs.shape
        nc = cdofs.shape[1]
        r = np.repeat(rdofs[:, :, None], nc, axis=2)
        c = np.repeat(cdofs[:, None, :], nr, axis=1)
        v = np.broadcast_to(Ke[None, :, :], (nt, nr, nc))
        if scale is not None:
            v = v * np.asarray(scale)[:, None, None]
        self.rows.append(r.ravel())
        self.cols.append(c.ravel())
        self.vals.append(np.ascontiguousarray(v).ravel())

    def tocsr(self):
        if not self.rows:
            return sp.csr_matrix((self.nr, self.nc))
        return sp.coo_matrix((np.concatenate(self.vals), (np.concatenate(self.rows), np.concatenate(self.cols))),
                             shape=(self.nr, self.nc)).tocsr()


# =====================================================================
# grid transfer (Sec. 3.3)
# =====================================================================
def _kuhn_locate(y, cdims):
    """Coarse cube and barycentric coordinates of points y given in coarse
    lattice units: the containing Kuhn tetrahedron of the cube."""
    cdims = np.asarray(cdims)
    q = np.clip(np.floor(y).astype(np.int64), 0, cdims[None, :] - 1)
    t = y - q
    perm = np.argsort(-t, axis=1, kind="stable")                       # descending coordinates
    ts = np.take_along_axis(t, perm, axis=1)
    lmb = np.stack([1 - ts[:, 0], ts[:, 0] - ts[:, 1], ts[:, 1] - ts[:, 2], ts[:, 2]], axis=1)
    # vertices of the tetrahedron along the path 0 -> e_p0 -> e_p0+e_p1 -> 1
    verts = np.zeros((y.shape[0], 4, 3), dtype=np.int64)
    verts[:, 0] = q
    cur = q.copy()
    for s in range(3):
        cur = cur.copy()
        cur[np.arange(y.shape[0]), perm[:, s]] += 1
        verts[:, s + 1] = cur
    return verts, lmb


def prolongation_matrix(fine: Lattice, coarse: Lattice, order):
    """I_{l-1}^l: evaluation of the coarse P1/P2 basis at the fine nodes."""
    if order == 1:
        Yf = fine.p1_int_coords().astype(np.float64) / 2.0
        verts, lmb = _kuhn_locate(Yf, coarse.dims)
        vals = fe.basis_values(lmb, 1)
        cols = coarse.p1_index(verts)
        nf, nc = fine.p1_count(), coarse.p1_count()
    else:
        Yf = fine.p2_int_coords().astype(np.float64) / 4.0
        verts, lmb = _kuhn_locate(Yf, coarse.dims)
        vals = fe.basis_values(lmb, 2)
        pos = [2 * verts[:, a] for a in range(4)] + [verts[:, a] + verts[:, b] for a, b in fe.EDGES]
        cols = np.stack([coarse.p2_index(v) for v in pos], axis=1)
        nf, nc = fine.p2_count(), coarse.p2_count()
    rows = np.repeat(np.arange(nf)[:, None], cols.shape[1], axis=1)
    keep = np.abs(vals) > 1e-14
    P = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(nf, nc)).tocsr()
    return P


# =====================================================================
# the hierarchy, coarse solve, V-cycle and FMG (Algorithm 1)
# =====================================================================
class StokesHierarchy:
    def __init__(self, box, H, L, disc, coarse_level=0, nu_a=0.0, pspg_rhs=True, workload=None,
                 gs_order="multicolour"):
        self.box, self.H, self.L, self.disc, self.lc = tuple(box), H, L, disc, coarse_level
        self.lv = {l: StokesLevel(box, H, l, disc, nu_a, pspg_rhs) for l in range(coarse_level, L + 1)}
        for lev in self.lv.values():
            lev.set_gs_order(gs_order)
        self.order_v = self.lv[L].order_v
        self.Pv, self.Pp = {}, {}
        for l in range(coarse_level + 1, L + 1):
            self.Pv[l] = prolongation_matrix(self.lv[l].lat, self.lv[l - 1].lat, self.order_v)
            self.Pp[l] = prolongation_matrix(self.lv[l].lat, self.lv[l - 1].lat, 1)
        self._coarse = None
        self.rhs, self.W = {}, {}
        if workload is not None:
            self.set_workload(workload)

    def set_workload(self, workload):
        self.workload = workload
        for l, lev in self.lv.items():
            self.rhs[l], self.W[l] = lev.assemble_rhs(workload)

    # ------------------------------------------------------------ transfers
    def prolongate(self, l, xc):
        """Correction prolongation I_{l-1}^l (velocity Dirichlet rows stay 0)."""
        fine, coarse = self.lv[l], self.lv[l - 1]
        uc, pc = coarse.split(xc)
        uf = [np.where(fine.vint, self.Pv[l] @ uc[c], 0.0) for c in range(3)]
        return fine.join(uf, self.Pp[l] @ pc)

    def restrict(self, l, rf):
        """I_l^{l-1} = (I_{l-1}^l)^T; coarse Dirichlet velocity rows zeroed."""
        fine, coarse = self.lv[l], self.lv[l - 1]
        uf, pf = fine.split(rf)
        uc = [np.where(coarse.vint, self.Pv[l].T @ uf[c], 0.0) for c in range(3)]
        return coarse.join(uc, self.Pp[l].T @ pf)

    def fmg_interpolate(self, l, xc):
        """FMG interpolation of the full coarse solution (boundary values w
        included), then the fine Dirichlet rows are reset to the lifting form."""
        fine, coarse = self.lv[l], self.lv[l - 1]
        uc, pc = coarse.split(xc + self.W[l - 1])
        uf = [np.where(fine.vint, self.Pv[l] @ uc[c], 0.0) for c in range(3)]
        return fine.join(uf, self.Pp[l] @ pc)

    # --------------------------------------------------------- coarse solve
    def coarse_matrix(self):
        lev = self.lv[self.lc]
        I = np.nonzero(lev.vint)[0]
        A = lev.A[I][:, I].toarray()
        Bs = [lev.B[c][:, I].toarray() for c in range(3)]
        nI, npp = len(I), lev.np
        n = 3 * nI + npp
        K = np.zeros((n + 1, n + 1))
        for c in range(3):
            K[c * nI:(c + 1) * nI, c * nI:(c + 1) * nI] = A
            K[c * nI:(c + 1) * nI, 3 * nI:n] = Bs[c].T
            K[3 * nI:n, c * nI:(c + 1) * nI] = Bs[c]
        K[3 * nI:n, 3 * nI:n] = -lev.C.toarray()
        K[3 * nI:n, n] = lev.ML
        K[n, 3 * nI:n] = lev.ML
        return K, I

    def coarse_solve(self, b):
        """Direct solve of calA_c x = b with int p_h = 0 (bordered system)."""
        lev = self.lv[self.lc]
        if self._coarse is None:
            self._coarse = self.coarse_matrix()
        K, I = self._coarse
        nI = len(I)
        u, p = lev.split(b)
        rhs = np.concatenate([u[0][I], u[1][I], u[2][I], p, [0.0]])
        sol = np.linalg.solve(K, rhs)
        x = np.zeros(lev.size)
        xu, xp = lev.split(x)
        for c in range(3):
            xu[c][I] = sol[c * nI:(c + 1) * nI]
        xp[:] = sol[3 * nI:3 * nI + lev.np]
        return x

    # ---------------------------------------------------------------- cycles
    def vcycle(self, lf, l, x, b, prm: Params):
        """VAR-V-CYCLE of Algorithm 1."""
        if l == self.lc:
            return self.coarse_solve(b)
        lev = self.lv[l]
        for _ in range(prm.nu_pre + (lf - l) * prm.nu_inc):
            x = lev.uzawa(x, b, prm)
        r = lev.residual(x, b)
        rc = self.restrict(l, r)
        xc = self.vcycle(lf, l - 1, np.zeros(self.lv[l - 1].size), rc, prm)
        x = x + self.prolongate(l, xc)
        for _ in range(prm.nu_post + (lf - l) * prm.nu_inc):
            x = lev.uzawa(x, b, prm)
        return x

    def fmg(self, prm: Params, L=None):
        """FMG of Algorithm 1 up to level L; p projected to mean zero after
        the coarse solve and after every V-cycle."""
        L = self.L if L is None else L
        x = self.lv[self.lc].project_pressure(self.coarse_solve(self.rhs[self.lc]))
        for l in range(self.lc + 1, L + 1):
            x = self.fmg_interpolate(l, x)
            for _ in range(prm.kappa):
                x = self.lv[l].project_pressure(self.vcycle(l, l, x, self.rhs[l], prm))
        return x

    def solve_to_tolerance(self, prm: Params, eps=1e-12, rel=1e-12, max_cycles=200, x0=None):
        """Discrete solution x_l with ||r_u||_2, ||r_p||_2 < eps (Sec. 5.1)."""
        L = self.L
        lev = self.lv[L]
        b = self.rhs[L]
        x = self.fmg(prm) if x0 is None else x0.copy()
        bn = max(lev.norms(b))
        for it in range(max_cycles):
            ru, rp = lev.norms(lev.residual(x, b))
            if max(ru, rp) < max(eps, 0.0) and max(ru, rp) <= rel * bn + eps:
                return x, it
            x = lev.project_pressure(self.vcycle(L, L, x, b, prm))
        return x, max_cycles

    # ---------------------------------------------------------------- errors
    def error_norms(self, x, l=None, exact_level=None):
        """||e(x)||_2 of Eq. error: M-norm on level l+1 of x* - I x, velocity
        and pressure separately, pressures compared with zero mean."""
        l = self.L if l is None else l
        fine = StokesLevel(self.box, self.H, l + 1, self.disc) if exact_level is None else exact_level
        coarse = self.lv[l]
        Pv = prolongation_matrix(fine.lat, coarse.lat, self.order_v)
        Pp = prolongation_matrix(fine.lat, coarse.lat, 1)
        uc, pc = coarse.split(x + self.W[l])
        Xv, Xp = fine.vcoords(), fine.pcoords()
        ue = self.workload.exact_velocity(Xv)
        pe = self.workload.exact_pressure(Xp)
        du = [ue[:, c] - Pv @ uc[c] for c in range(3)]
        pi = Pp @ pc
        pe = pe - np.dot(fine.ML, pe) / fine.ML.sum()
        pi = pi - np.dot(fine.ML, pi) / fine.ML.sum()
        dp = pe - pi
        eu = np.sqrt(sum(d @ (fine.Mv @ d) for d in du))
        ep = np.sqrt(dp @ (fine.Mp @ dp))
        return float(eu), float(ep)

    # ------------------------------------------------------- omega estimate
    def estimate_omega_inv(self, v0, iters=100, l=None):
        """Largest eigenvalue of M_L^{-1} (C + B A_s^{-1} B^T) (Eq.
        omega-eigenvalue-problem) by power iteration; A_s^{-1} is one
        symmetric GS sweep from a zero guess.  v0: start vector (input)."""
        l = self.L if l is None else l
        lev = self.lv[l]
        v = v0 - np.dot(lev.ML, v0) / lev.ML.sum()
        v = v / np.linalg.norm(v)
        lam_est = 0.0
        for _ in range(iters):
            z = [np.where(lev.vint, lev.B[c].T @ v, 0.0) for c in range(3)]
            y = []
            for c in range(3):
                yc = np.zeros(lev.nv)
                lev.gs_sweep(yc, z[c], backward=False)
                lev.gs_sweep(yc, z[c], backward=True)
                y.append(yc)
            w = (lev.C @ v + sum(lev.B[c] @ y[c] for c in range(3))) / lev.ML_hat
            lam_est = float(np.linalg.norm(w))
            v = w / lam_est
        return lam_est
