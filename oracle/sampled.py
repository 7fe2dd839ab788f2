"""Single rows of the Stokes operator computed from their definition (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For problem sizes where assembling global matrices is too expensive, a row
(calA x)_i of Eq. stokes-discrete is evaluated directly: loop over the micro
tetrahedra T of the Kuhn lattice that contain DoF i, add the element
contributions K_T[i, :] x_T (oracle/fe.py element matrices; with a variable
viscosity, scaled by nu_T at the centroid).  Dirichlet velocity rows are 0.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

from . import fe
from .mesh import PERMS, Lattice

_ELEM = {}


def _class_mats(order, h, s):
    key = (order, h, s)
    if key not in _ELEM:
        v = np.zeros(3, dtype=np.int64)
        verts = [v.copy()]
        for d in PERMS[s]:
            v[d] += 1
            verts.append(v.copy())
        X = np.array(verts, dtype=np.float64) * h
        _ELEM[key] = (np.array(verts), fe.stiffness(X, order), fe.divergence(X, order), fe.pspg(X),
                      fe.mass(X, order), fe.mass(X, 1))
    return _ELEM[key]


def _tet_dofs(base, verts, order, lat):
    """Velocity and pressure DoF indices (canonical) of the tet at cube base."""
    V = verts + base[None, :]
    pd = lat.p1_index(V)
    if order == 1:
        return pd, pd
    pos = [2 * V[a] for a in range(4)] + [V[a] + V[b] for a, b in fe.EDGES]
    return np.array([lat.p2_index(p) for p in pos]), pd


def sample_rows(box, H, level, disc, x, rows, nu_a=0.0, with_abs=False):
    """rows: list of (field, canonical node index), field 0..2 velocity, 3
    pressure.  x: canonical block vector.  Returns the values (calA x)_row
    (and, with with_abs, the sums of |a_ij x_j| that bound their rounding)."""
    lat = Lattice(box, H, level)
    order = 1 if disc == "P1P1" else 2
    nv = lat.p1_count() if order == 1 else lat.p2_count()
    u = [x[c * nv:(c + 1) * nv] for c in range(3)]
    p = x[3 * nv:]
    dims = np.array(lat.dims)
    out, absout = [], []
    for field, node in rows:
        if field < 3:
            IJK = lat.p1_int_coords_of(node) if order == 1 else lat.p2_int_coords_of(node)
            twice = IJK * (2 if order == 1 else 1)          # doubled-lattice position
            lim = 2 * dims
            if np.any(twice == 0) or np.any(twice == lim):
                out.append(0.0)
                absout.append(0.0)
                continue
        else:
            twice = lat.p1_int_coords_of(node) * 2
        lo = np.maximum((twice - 2) // 2, 0)
        hi = np.minimum(twice // 2, dims - 1)
        val = 0.0
        aval = 0.0
        for cz, cy, cx in itertools.product(*(range(lo[d], hi[d] + 1) for d in (2, 1, 0))):
            base = np.array([cx, cy, cz])
            for s in range(6):
                verts, K, D, Cm, _, _ = _class_mats(order, lat.h, s)
                vd, pd = _tet_dofs(base, verts, order, lat)
                cent_z = (verts[:, 2].mean() + cz) * lat.h
                nuT = math.exp(nu_a * cent_z)
                if field < 3:
                    hit = np.nonzero(vd == node)[0]
                    if hit.size == 0:
                        continue
                    a = hit[0]
                    val += nuT * K[a] @ u[field][vd] + D[field][:, a] @ p[pd]
                    aval += nuT * np.abs(K[a]) @ np.abs(u[field][vd]) + np.abs(D[field][:, a]) @ np.abs(p[pd])
                else:
                    hit = np.nonzero(pd == node)[0]
                    if hit.size == 0:
                        continue
                    k = hit[0]
                    val += sum(D[c][k] @ u[c][vd] for c in range(3))
                    aval += sum(np.abs(D[c][k]) @ np.abs(u[c][vd]) for c in range(3))
                    if order == 1:
                        val -= (Cm[k] @ p[pd]) / nuT
                        aval += (np.abs(Cm[k]) @ np.abs(p[pd])) / nuT
        out.append(val)
        absout.append(aval)
    return (np.array(out), np.array(absout)) if with_abs else np.array(out)
