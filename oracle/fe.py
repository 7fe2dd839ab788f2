"""Element matrices on a single tetrahedron, computed exactly (oracle).

TEST INFRASTRUCTURE ONLY: the oracle is imported by tests, by the smoke check
and by the benchmark's CPU-baseline leg, never by the CUDA product path.

Every integrand is a polynomial in the barycentric coordinates lambda_0..3 of
the tetrahedron T, integrated with the closed form

    int_T lambda_0^a0 lambda_1^a1 lambda_2^a2 lambda_3^a3 dx
        = 6 |T| a0! a1! a2! a3! / (a0 + a1 + a2 + a3 + 3)!

so the matrices are exact up to rounding.

Bilinear forms (Sec. 2, Eq. stokes-weak / stokes-discrete / pspg):
  * stiffness   a_ij = int grad phi_i . grad phi_j
  * divergence  b_kj^(d) = - int psi_k d_d phi_j           (psi: P1 pressure)
  * mass        m_ij = int phi_i phi_j
  * PSPG        c_kl = delta_T h_T^2 int grad psi_k . grad psi_l,
                h_T = |T|^(1/3), delta_T = 1/12
  * PSPG load   l_kj^(d) = - delta_T h_T^2 int (d_d psi_k) phi_j   (consistent
                stabilisation of the continuity equation with the interpolated
                forcing f_h = sum_j f(x_j) phi_j)
P2 local numbering: vertices 0..3, then edges (0,1),(0,2),(0,3),(1,2),(1,3),(2,3).
"""
from __future__ import annotations

import math
from collections import defaultdict

import numpy as np

EDGES = [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]
PSPG_DELTA = 1.0 / 12.0


# -------------------------------------------------------------- polynomials
def _mono(*exps):
    return tuple(exps)


def poly_mul(p, q):
    out = defaultdict(float)
    for ea, ca in p.items():
        for eb, cb in q.items():
            out[tuple(a + b for a, b in zip(ea, eb))] += ca * cb
    return dict(out)


def poly_diff(p, i):
    """Partial derivative with respect to lambda_i (lambda treated as free)."""
    out = defaultdict(float)
    for e, c in p.items():
        if e[i] > 0:
            ne = list(e)
            ne[i] -= 1
            out[tuple(ne)] += c * e[i]
    return dict(out)


def poly_integrate(p, vol):
    total = 0.0
    for e, c in p.items():
        num = 1
        for a in e:
            num *= math.factorial(a)
        total += c * 6.0 * vol * num / math.factorial(sum(e) + 3)
    return total


def lam(i):
    e = [0, 0, 0, 0]
    e[i] = 1
    return {tuple(e): 1.0}


def p1_basis():
    return [lam(i) for i in range(4)]


def p2_basis():
    basis = []
    for i in range(4):
        e2 = [0, 0, 0, 0]
        e2[i] = 2
        basis.append({tuple(e2): 2.0, tuple(lam(i).keys())[0]: -1.0})
    for (i, j) in EDGES:
        e = [0, 0, 0, 0]
        e[i] += 1
        e[j] += 1
        basis.append({tuple(e): 4.0})
    return basis


# ---------------------------------------------------------------- geometry
def tet_geometry(X):
    """X: (4,3) vertex coordinates.  Returns (volume, grad_lambda (4,3))."""
    X = np.asarray(X, dtype=np.float64)
    J = np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)  # columns
    vol = abs(np.linalg.det(J)) / 6.0
    Jinv = np.linalg.inv(J)          # lambda_{1..3} = Jinv (x - X0)
    g = np.zeros((4, 3))
    g[1:] = Jinv
    g[0] = -Jinv.sum(axis=0)
    return vol, g


def _grad_coeffs(basis):
    """For each basis function, its list of d phi / d lambda_i polynomials."""
    return [[poly_diff(b, i) for i in range(4)] for b in basis]


_CACHE = {}


def _basis(order):
    if order not in _CACHE:
        b = p1_basis() if order == 1 else p2_basis()
        _CACHE[order] = (b, _grad_coeffs(b))
    return _CACHE[order]


# ---------------------------------------------------------- element matrices
def stiffness(X, order):
    vol, g = tet_geometry(X)
    G = g @ g.T
    basis, dphi = _basis(order)
    n = len(basis)
    K = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            s = 0.0
            for i in range(4):
                for j in range(4):
                    if G[i, j] == 0.0:
                        continue
                    s += G[i, j] * poly_integrate(poly_mul(dphi[a][i], dphi[b][j]), vol)
            K[a, b] = s
    return K


def mass(X, order):
    vol, _ = tet_geometry(X)
    basis, _ = _basis(order)
    n = len(basis)
    M = np.zeros((n, n))
    for a in range(n):
        for b in range(n):
            M[a, b] = poly_integrate(poly_mul(basis[a], basis[b]), vol)
    return M


def divergence(X, order):
    """D[d] (4 x n): D[d][k, j] = -int psi_k d_d phi_j, psi_k = lambda_k."""
    vol, g = tet_geometry(X)
    basis, dphi = _basis(order)
    n = len(basis)
    D = np.zeros((3, 4, n))
    for k in range(4):
        for j in range(n):
            for i in range(4):
                val = poly_integrate(poly_mul(lam(k), dphi[j][i]), vol)
                D[:, k, j] -= g[i] * val
    return D


def pspg(X, delta=PSPG_DELTA):
    vol, g = tet_geometry(X)
    hT2 = vol ** (2.0 / 3.0)
    return delta * hT2 * vol * (g @ g.T)


def pspg_load(X, order, delta=PSPG_DELTA):
    """L[d] (4 x n): L[d][k, j] = -delta h_T^2 (d_d psi_k) int phi_j."""
    vol, g = tet_geometry(X)
    hT2 = vol ** (2.0 / 3.0)
    basis, _ = _basis(order)
    intphi = np.array([poly_integrate(b, vol) for b in basis])
    L = np.zeros((3, 4, len(basis)))
    for d in range(3):
        L[d] = -delta * hT2 * np.outer(g[:, d], intphi)
    return L


def basis_values(lmb, order):
    """Values of the P1 or P2 basis at barycentric points lmb (N, 4)."""
    lmb = np.asarray(lmb, dtype=np.float64)
    if order == 1:
        return lmb.copy()
    out = np.zeros((lmb.shape[0], 10))
    for i in range(4):
        out[:, i] = lmb[:, i] * (2.0 * lmb[:, i] - 1.0)
    for e, (i, j) in enumerate(EDGES):
        out[:, 4 + e] = 4.0 * lmb[:, i] * lmb[:, j]
    return out
