"""Stokes operators on Bey-refined unstructured macro meshes (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 2 and Sec. 2.1: every macro tetrahedron of T_0 is refined uniformly by
Bey's rule, and the refined mesh is the union of the refined macro
tetrahedra with the nodes on shared faces, edges and vertices identified.
The blocks of Eq. stokes-discrete (A, B, C and the masses) are assembled
element by element from the exact element matrices of fe.py on every micro
tetrahedron of that mesh, for any conforming macro mesh -- the paper's cube
of 24 macro tetrahedra (Sec. 5.1.1) included, whose refinement is not one
lattice.  Constant viscosity only.

Node numbering: the P1 nodes are the mesh vertices and the P2 nodes the
vertices plus the edge midpoints, each set ordered by (z, y, x) with x
fastest -- on a Kuhn box this is the lexicographic numbering of
oracle/mesh.py, so the two assemblies can be compared entry by entry.
Velocity Dirichlet nodes are the nodes on the boundary faces of the refined
mesh (faces of exactly one tetrahedron).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

from . import fe
from .mesh import bey_refine


def _numbering(points, scale):
    """(node index of each point, node coordinates): points keyed on the
    dyadic grid of spacing 1/scale, nodes ordered by (z, y, x)."""
    keys = np.rint(points * scale).astype(np.int64)
    uniq, inv = np.unique(keys[:, ::-1], axis=0, return_inverse=True)
    return inv.reshape(-1), uniq[:, ::-1].astype(np.float64) / scale


def _assemble(nr, nc, rows, cols, mats):
    """sum over tetrahedra T of P_T^T K_T P_T (rows, cols: (nt, k) DoF
    indices, mats: (nt, k_r, k_c) element matrices)."""
    r = np.repeat(rows[:, :, None], cols.shape[1], axis=2).ravel()
    c = np.repeat(cols[:, None, :], rows.shape[1], axis=1).ravel()
    return sp.coo_matrix((np.asarray(mats).ravel(), (r, c)), shape=(nr, nc)).tocsr()


class UnstructuredLevel:
    """Level `level` of a macro mesh (verts (nv, 3), tets (nt, 4) vertex
    indices) for disc = "P1P1" (PSPG) or "P2P1" (Taylor-Hood)."""

    def __init__(self, verts, tets, level, disc):
        self.disc = disc
        self.order_v = 1 if disc == "P1P1" else 2
        X = np.array(bey_refine(verts, tets, level), dtype=np.float64)       # (nt, 4, 3)
        self.nt = X.shape[0]
        scale = 2.0 ** (level + 3)                                         # holds every edge midpoint
        pidx, self.pcoords = _numbering(X.reshape(-1, 3), scale)
        tet_p = pidx.reshape(self.nt, 4)
        if self.order_v == 1:
            tet_v, self.vcoords = tet_p, self.pcoords
        else:
            mids = np.stack([(X[:, a] + X[:, b]) / 2.0 for a, b in fe.EDGES], axis=1)   # (nt, 6, 3)
            allp = np.concatenate([X, mids], axis=1).reshape(-1, 3)
            vidx, self.vcoords = _numbering(allp, scale)
            tet_v = vidx.reshape(self.nt, 10)
        self.np, self.nv = self.pcoords.shape[0], self.vcoords.shape[0]
        self.tet_v, self.tet_p = tet_v, tet_p

        K, Mv, D, Cm, Mp = [], [], [[], [], []], [], []
        for t in range(self.nt):
            Xt = X[t]
            K.append(fe.stiffness(Xt, self.order_v))
            Mv.append(fe.mass(Xt, self.order_v))
            De = fe.divergence(Xt, self.order_v)
            for d in range(3):
                D[d].append(De[d])
            Cm.append(fe.pspg(Xt) if disc == "P1P1" else np.zeros((4, 4)))
            Mp.append(fe.mass(Xt, 1))
        self.A = _assemble(self.nv, self.nv, tet_v, tet_v, K)
        self.Mv = _assemble(self.nv, self.nv, tet_v, tet_v, Mv)
        self.B = [_assemble(self.np, self.nv, tet_p, tet_v, D[d]) for d in range(3)]
        self.C = _assemble(self.np, self.np, tet_p, tet_p, Cm)
        self.Mp = _assemble(self.np, self.np, tet_p, tet_p, Mp)

        # boundary faces: faces of exactly one tetrahedron; their vertices
        # (and, for P2, their edge midpoints) are the Dirichlet nodes
        count = {}
        for t in range(self.nt):
            for f in itertools.combinations(range(4), 3):
                key = tuple(sorted(tet_p[t, list(f)]))
                count[key] = count.get(key, 0) + 1
        bnd_p = np.zeros(self.np, dtype=bool)
        bfaces = [f for f, m in count.items() if m == 1]
        for f in bfaces:
            bnd_p[list(f)] = True
        if self.order_v == 1:
            self.vbnd = bnd_p
        else:
            # a P2 node lies on the boundary iff it is a vertex of a boundary
            # face or the midpoint of one of its edges
            vbnd = np.zeros(self.nv, dtype=bool)
            bset = set(bfaces)
            loc = {e: 4 + q for q, e in enumerate(fe.EDGES)}
            for t in range(self.nt):
                for f in itertools.combinations(range(4), 3):
                    if tuple(sorted(tet_p[t, list(f)])) in bset:
                        vbnd[tet_v[t, list(f)]] = True
                        for a, b in itertools.combinations(f, 2):
                            vbnd[tet_v[t, loc[(a, b)]]] = True
            self.vbnd = vbnd
        self.vint = ~self.vbnd

    @property
    def size(self):
        return 3 * self.nv + self.np

    def split(self, x):
        return [x[c * self.nv:(c + 1) * self.nv] for c in range(3)], x[3 * self.nv:]

    def join(self, u, p):
        return np.concatenate(list(u) + [p])

    def apply(self, x):
        """y = calA x (Eq. stokes-discrete); Dirichlet velocity rows are 0."""
        u, p = self.split(x)
        yu = [np.where(self.vint, self.A @ u[c] + self.B[c].T @ p, 0.0) for c in range(3)]
        yp = sum(self.B[c] @ u[c] for c in range(3)) - self.C @ p
        return self.join(yu, yp)
