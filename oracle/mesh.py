"""Refined meshes T_l of Kuhn-box macro meshes (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2 and Sec. 2.1: each macro tetrahedron of T_0 is refined uniformly
(Bey's algorithm) l times.  For a macro mesh made of Kuhn-split cubes of side
H whose tetrahedra list their vertices along the cube's monotone path, the
refined mesh on level l is the Kuhn (Freudenthal) lattice with spacing
h = H / 2^l: every micro-cube of the lattice is split into the 6 tetrahedra
{0, e_s0, e_s0 + e_s1, (1,1,1)} for the 6 permutations s.  ``bey_refine``
below implements Bey's rule so that the tests can check this identity
instead of assuming it.

Node sets used by the oracle:
  * P1 nodes: lattice points (i, j, k), 0 <= i <= nx, ...
  * P2 nodes: points of the doubled lattice (I, J, K), 0 <= I <= 2 nx, ...
    (vertex DoFs at even points, edge-midpoint DoFs elsewhere; Sec. 2.2)
Node numbering is lexicographic with the first index fastest.
"""
from __future__ import annotations

import itertools

import numpy as np

PERMS = list(itertools.permutations(range(3)))   # the 6 Kuhn classes


class Lattice:
    """Level-l Kuhn lattice of an (mx, my, mz) box of cubes with side H."""

    def __init__(self, box, H, level):
        self.box = tuple(int(b) for b in box)
        self.H = float(H)
        self.level = int(level)
        n = 2 ** self.level
        self.n = n
        self.dims = tuple(b * n for b in self.box)          # cells per direction
        self.h = self.H / n

    # ---- P1 / pressure nodes
    def p1_shape(self):
        return tuple(d + 1 for d in self.dims)

    def p1_count(self):
        nx, ny, nz = self.p1_shape()
        return nx * ny * nz

    def p1_index(self, ijk):
        ijk = np.asarray(ijk)
        nx, ny, _ = self.p1_shape()
        return ijk[..., 0] + nx * (ijk[..., 1] + ny * ijk[..., 2])

    def p1_coords(self):
        nx, ny, nz = self.p1_shape()
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1) * self.h

    def p1_int_coords(self):
        nx, ny, nz = self.p1_shape()
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def p1_int_coords_of(self, index):
        """(i, j, k) of one P1 node index (the inverse of p1_index)."""
        nx, ny, _ = self.p1_shape()
        index = int(index)
        return np.array([index % nx, (index // nx) % ny, index // (nx * ny)], dtype=np.int64)

    # ---- P2 nodes (doubled lattice)
    def p2_shape(self):
        return tuple(2 * d + 1 for d in self.dims)

    def p2_count(self):
        a, b, c = self.p2_shape()
        return a * b * c

    def p2_index(self, IJK):
        IJK = np.asarray(IJK)
        a, b, _ = self.p2_shape()
        return IJK[..., 0] + a * (IJK[..., 1] + b * IJK[..., 2])

    def p2_int_coords(self):
        a, b, c = self.p2_shape()
        k, j, i = np.meshgrid(np.arange(c), np.arange(b), np.arange(a), indexing="ij")
        return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)

    def p2_int_coords_of(self, index):
        """(I, J, K) of one P2 node index (the inverse of p2_index)."""
        a, b, _ = self.p2_shape()
        index = int(index)
        return np.array([index % a, (index // a) % b, index // (a * b)], dtype=np.int64)

    def p2_coords(self):
        return self.p2_int_coords() * (0.5 * self.h)

    # ---- micro tetrahedra
    def tets(self):
        """(ntets, 4, 3) integer lattice coordinates of the micro-tet vertices,
        and (ntets,) Kuhn class ids; cube-major order."""
        nx, ny, nz = self.dims
        k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)       # (ncubes, 3)
        out = np.zeros((base.shape[0], 6, 4, 3), dtype=np.int64)
        cls = np.zeros((base.shape[0], 6), dtype=np.int64)
        for s, perm in enumerate(PERMS):
            v = base.copy()
            out[:, s, 0] = v
            for step, d in enumerate(perm):
                v = v.copy()
                v[:, d] += 1
                out[:, s, step + 1] = v
            cls[:, s] = s
        return out.reshape(-1, 4, 3), cls.reshape(-1)

    def boundary_mask_p1(self):
        ijk = self.p1_int_coords()
        dims = np.array(self.dims)
        return np.any((ijk == 0) | (ijk == dims[None, :]), axis=1)

    def boundary_mask_p2(self):
        IJK = self.p2_int_coords()
        dims = 2 * np.array(self.dims)
        return np.any((IJK == 0) | (IJK == dims[None, :]), axis=1)


# ----------------------------------------------------------- Bey refinement
def bey_children(t):
    """Bey's uniform refinement of the tetrahedron t = (x0, x1, x2, x3)
    (Sec. 2, Fig. hhg-refinement): four corner children and four children
    of the inner octahedron, all sharing the diagonal x02 -- x13."""
    x0, x1, x2, x3 = t
    m = lambda a, b: tuple((np.asarray(a) + np.asarray(b)) / 2.0)
    x01, x02, x03 = m(x0, x1), m(x0, x2), m(x0, x3)
    x12, x13, x23 = m(x1, x2), m(x1, x3), m(x2, x3)
    return [
        (x0, x01, x02, x03), (x01, x1, x12, x13), (x02, x12, x2, x23), (x03, x13, x23, x3),
        (x01, x02, x03, x13), (x01, x02, x12, x13), (x02, x03, x13, x23), (x02, x12, x13, x23),
    ]


def bey_refine(macro_verts, macro_tets, level):
    """Refine every macro tetrahedron ``level`` times with Bey's rule."""
    tets = [tuple(tuple(float(c) for c in macro_verts[v]) for v in t) for t in macro_tets]
    for _ in range(level):
        nxt = []
        for t in tets:
            nxt.extend(bey_children(t))
        tets = nxt
    return tets
