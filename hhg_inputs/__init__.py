"""Seeded and closed-form synthetic inputs for the Stokes workloads.

This module is shared by the CUDA path's tests/benchmark and by the CPU
oracle.  It holds *inputs only*: macro meshes given as vertex/tetrahedron
lists, closed-form velocity/pressure/forcing fields evaluated at points, and
seeded random parameters.  It contains none of the discretisation or solver
arithmetic (no element matrices, no stencils, no smoothing, no transfers).

Workloads (all in the paper's setting of an all-Dirichlet cube, Sec. 2 and
Sec. 5.1.1):
  * ``curl``   -- u = curl(psi, psi, psi) with psi = sin(pi x) sin(pi y) sin(pi z),
                  p = x + y + z - 1.5 on the unit cube; forcing for the
                  constant-coefficient Stokes system (Eq. stokes-cc) or for the
                  variable-viscosity form -div(nu grad u_c) + d_c p = f_c with
                  nu = exp(a z).
  * ``paper``  -- the analytic cube solution of Sec. 5.1.1 (u = (-4 cos 4z,
                  8 cos 8x, -2 cos 2y), p = sin 4x sin 8y sin 2z + const).
  * ``modes``  -- random smooth forcing: per component a sum of 8 sine modes
                  with random integer wave vectors, phases and N(0,1) amplitudes,
                  zero Dirichlet data (batched workload).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

PI = math.pi


# ---------------------------------------------------------------------------
# macro meshes (coarse grid T_0 of Sec. 2): unions of Kuhn-split unit cubes
# ---------------------------------------------------------------------------
def kuhn_box_macro_mesh(mx: int, my: int, mz: int, H: float = 1.0):
    """Macro mesh of an mx x my x mz box of cubes with side H, each cube split
    into the 6 tetrahedra around its (0,0,0)-(1,1,1) diagonal.

    Returns (verts (nv,3) float64, tets (nt,4) int32).  Every tetrahedron's
    vertices are listed along its monotone path 0 -> e_a -> e_a+e_b -> 1 of
    the cube, i.e. in Kuhn order.
    """
    nxv, nyv = mx + 1, my + 1
    verts = np.array([[i * H, j * H, k * H]
                      for k in range(mz + 1) for j in range(my + 1) for i in range(mx + 1)],
                     dtype=np.float64)

    def vid(i, j, k):
        return i + nxv * (j + nyv * k)

    tets = []
    for k in range(mz):
        for j in range(my):
            for i in range(mx):
                for perm in itertools.permutations(range(3)):
                    v = [i, j, k]
                    path = [tuple(v)]
                    for d in perm:
                        v[d] += 1
                        path.append(tuple(v))
                    tets.append([vid(*q) for q in path])
    return verts, np.array(tets, dtype=np.int32)


def cube24_macro_mesh():
    """The unit cube as 24 macro tetrahedra: the cube's 8 corners, its 6 face
    centres and its centre; every face is cut into 4 triangles (two adjacent
    corners and the face centre), each the base of one tetrahedron with apex at
    the cube centre.  Not a Kuhn box (its refinement is not one lattice).

    Returns (verts (15,3) float64, tets (24,4) int32)."""
    corners = [(i, j, k) for k in (0, 1) for j in (0, 1) for i in (0, 1)]
    verts = [tuple(float(c) for c in v) for v in corners]
    tets = []
    for d in range(3):
        for side in (0.0, 1.0):
            fc = [0.5, 0.5, 0.5]
            fc[d] = side
            verts.append(tuple(fc))
            f = len(verts) - 1
            # the face's corners in cyclic order around it
            a, b = [e for e in range(3) if e != d]
            ring = []
            for ua, ub in ((0, 0), (1, 0), (1, 1), (0, 1)):
                v = [0.0, 0.0, 0.0]
                v[d], v[a], v[b] = side, float(ua), float(ub)
                ring.append(verts.index(tuple(v)))
            for q in range(4):
                tets.append([ring[q], ring[(q + 1) % 4], f])
    verts.append((0.5, 0.5, 0.5))
    c = len(verts) - 1
    tets = [t + [c] for t in tets]
    return np.array(verts, dtype=np.float64), np.array(tets, dtype=np.int32)


# ---------------------------------------------------------------------------
# manufactured solution "curl" (divergence-free by construction)
# ---------------------------------------------------------------------------
def _psi_derivs(X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    sx, sy, sz = np.sin(PI * x), np.sin(PI * y), np.sin(PI * z)
    cx, cy, cz = np.cos(PI * x), np.cos(PI * y), np.cos(PI * z)
    psi = sx * sy * sz
    px, py, pz = PI * cx * sy * sz, PI * sx * cy * sz, PI * sx * sy * cz
    pxz = PI * PI * cx * sy * cz
    pyz = PI * PI * sx * cy * cz
    pzz = -PI * PI * psi
    return psi, px, py, pz, pxz, pyz, pzz


def curl_velocity(X):
    _, px, py, pz, _, _, _ = _psi_derivs(X)
    return np.stack([py - pz, pz - px, px - py], axis=1)


def curl_pressure(X, center=(0.5, 0.5, 0.5)):
    return X[:, 0] + X[:, 1] + X[:, 2] - float(sum(center))


def curl_forcing(X, nu_a: float = 0.0):
    """f = -div(nu grad u_c) + grad p for nu = exp(nu_a * z) (nu = 1 if nu_a = 0)."""
    psi, px, py, pz, pxz, pyz, pzz = _psi_derivs(X)
    u = np.stack([py - pz, pz - px, px - py], axis=1)
    nu = np.exp(nu_a * X[:, 2])
    dzu = np.stack([pyz - pzz, pzz - pxz, pxz - pyz], axis=1)
    # -nu * Laplace(u_c) = 3 pi^2 nu u_c ; -(d_z nu)(d_z u_c) = -a nu d_z u_c ; grad p = (1,1,1)
    return nu[:, None] * (3.0 * PI * PI * u) - (nu_a * nu)[:, None] * dzu + 1.0


def viscosity(X, nu_a: float):
    return np.exp(nu_a * X[:, 2])


# ---------------------------------------------------------------------------
# the analytic cube solution of Sec. 5.1.1
# ---------------------------------------------------------------------------
_PAPER_P_MEAN = ((1 - math.cos(4)) / 4) * ((1 - math.cos(8)) / 8) * ((1 - math.cos(2)) / 2)


def paper_velocity(X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return np.stack([-4 * np.cos(4 * z), 8 * np.cos(8 * x), -2 * np.cos(2 * y)], axis=1)


def paper_pressure(X):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return np.sin(4 * x) * np.sin(8 * y) * np.sin(2 * z) - _PAPER_P_MEAN


def paper_forcing(X, nu_a: float = 0.0):
    if nu_a != 0.0:
        raise ValueError("the analytic cube solution is for unit viscosity")
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return np.stack([
        -64 * np.cos(4 * z) + 4 * np.cos(4 * x) * np.sin(8 * y) * np.sin(2 * z),
        512 * np.cos(8 * x) + 8 * np.sin(4 * x) * np.cos(8 * y) * np.sin(2 * z),
        -8 * np.cos(2 * y) + 2 * np.sin(4 * x) * np.sin(8 * y) * np.cos(2 * z)], axis=1)


# ---------------------------------------------------------------------------
# random smooth forcing (batched workload)
# ---------------------------------------------------------------------------
def random_modes(seed: int, n_modes: int = 8, kmax: int = 4):
    """Per component: wave vectors k_m in {1..kmax}^3, phases U[0, 2pi),
    amplitudes N(0, 1).  Returns a dict of arrays (3, n_modes, ...)."""
    rng = np.random.default_rng(seed)
    k = rng.integers(1, kmax + 1, size=(3, n_modes, 3))
    phi = rng.uniform(0.0, 2 * PI, size=(3, n_modes))
    amp = rng.standard_normal(size=(3, n_modes))
    return {"k": k, "phi": phi, "amp": amp}


def modes_forcing(X, modes):
    out = np.zeros((X.shape[0], 3))
    for c in range(3):
        for m in range(modes["k"].shape[1]):
            arg = PI * (X @ modes["k"][c, m].astype(np.float64)) + modes["phi"][c, m]
            out[:, c] += modes["amp"][c, m] * np.sin(arg)
    return out


def zero_field(X):
    return np.zeros((X.shape[0], 3))


# ---------------------------------------------------------------------------
# workload registry
# ---------------------------------------------------------------------------
class Workload:
    """Closed-form data of one Stokes problem: forcing f, Dirichlet data w and
    (if known) the exact solution (u, p)."""

    def __init__(self, kind: str, nu_a: float = 0.0, seed: int = 0, box=(1, 1, 1), H: float = 1.0):
        self.kind, self.nu_a, self.seed, self.box, self.H = kind, float(nu_a), seed, tuple(box), H
        ext = np.array(box, dtype=np.float64) * H
        self.center = tuple(0.5 * ext)
        if kind == "modes":
            self.modes = random_modes(seed)

    def forcing(self, X):
        if self.kind == "curl":
            return curl_forcing(X, self.nu_a)
        if self.kind == "paper":
            return paper_forcing(X, self.nu_a)
        if self.kind == "modes":
            return modes_forcing(X, self.modes)
        raise ValueError(self.kind)

    def dirichlet(self, X):
        if self.kind == "curl":
            return curl_velocity(X)
        if self.kind == "paper":
            return paper_velocity(X)
        return zero_field(X)

    def has_exact(self):
        return self.kind in ("curl", "paper")

    def exact_velocity(self, X):
        return curl_velocity(X) if self.kind == "curl" else paper_velocity(X)

    def exact_pressure(self, X):
        return curl_pressure(X, self.center) if self.kind == "curl" else paper_pressure(X)


def draw_viscosity_exponent(seed: int = 0, lo: float = 0.0, hi: float = 4.0) -> float:
    """The exponent a of nu = exp(a z), drawn uniformly in [lo, hi] from a seed."""
    return float(np.random.default_rng(seed).uniform(lo, hi))


def batched_problem_list(seed: int = 0, n: int = 64, levels=(3, 6)):
    """The batched workload: n problems with Kuhn boxes (mx,my,mz) in {1,2}^3,
    levels uniform in [levels[0], levels[1]], discretisation P1-P1 or P2-P1
    with probability 1/2 each, and random smooth forcing seeded per problem."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        box = tuple(int(v) for v in rng.integers(1, 3, size=3))
        level = int(rng.integers(levels[0], levels[1] + 1))
        disc = "P1P1" if rng.uniform() < 0.5 else "P2P1"
        out.append({"box": box, "level": level, "disc": disc, "seed": 1000 + i})
    return out
