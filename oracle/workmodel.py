"""The paper's work-unit (WU) cost model (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Sec. 4: a stencil with n entries costs 2n operations; block costs per level
(Eqs. cost-block-p2p1-a/b/c, cost-block-p1p1-ab/c) use the inner-unknown
counts of Table 1, N_tet(v) = v (v+1) (v+2) / 6 (Eq. num-unknowns-tet), and
the stencil sizes of Table 2.  Relaxation: W(A_f) = W(A) = W(A_s) / 2;
W(P^{-1}) = xi W(A_hat) + W(B^T) + W(B) + W(C).  V-cycle bound (Eq.
bound-var-v-cycle): W* = 8/7 W(V_L^L) + 16/49 nu_inc W(P^{-1}) with
W(V_L^L) = (nu_pre + nu_post) W(P^{-1}) + W(calA); FMG (Eq. cost-var-fmg):
8 kappa / 7 W*.
"""
from __future__ import annotations

from fractions import Fraction


def n_tet(v):
    return v * (v + 1) * (v + 2) // 6


def table1_counts(level):
    """Unknowns of one refined tetrahedron per DoF group (Table 1):
    (inner, including boundary) for vertices, xyz-edges and other edges."""
    n = 2 ** level
    return {
        "vertices": (n_tet(n - 3), n_tet(n + 1)),
        "xyz-edges": (n_tet(n - 1), n_tet(n - 1)),
        "other-edges": (n_tet(n - 2), n_tet(n)),
    }


STENCIL_FROM_ALL_P2 = {"vertex": 65, "x": 27, "y": 19, "z": 27, "xy": 27, "xz": 19, "yz": 27, "xyz": 19}
STENCIL_FROM_VERTEX_P2 = {"vertex": 15, "x": 8, "y": 6, "z": 8, "xy": 8, "xz": 6, "yz": 8, "xyz": 6}


def block_work(disc, level):
    """Operation counts W(A), W(B), W(C) on level l in the interior of one
    macro tetrahedron (Sec. 4.1)."""
    n = 2 ** level
    if disc == "P2P1":
        other = sum(v for k, v in STENCIL_FROM_ALL_P2.items() if k not in ("vertex", "xyz"))   # 146
        WB = 3 * (2 * 65) * n_tet(n - 3)
        WA = 3 * ((2 * 65) * n_tet(n - 3) + (2 * other) * n_tet(n - 2) + (2 * 19) * n_tet(n - 1))
        WC = 0
    else:
        WA = WB = 3 * (2 * 15) * n_tet(n - 3)
        WC = (2 * 15) * n_tet(n - 3)
    return WA, WB, WC


def normalized_blocks(disc, level=None):
    """(W(A), W(B), W(C)) / W(calA) at a level, or the l -> infinity limit
    (ratio of the leading n^3 coefficients) when level is None."""
    if level is None:
        if disc == "P2P1":
            WA = Fraction(3 * (130 + 2 * 146 + 38))
            WB = Fraction(3 * 130)
            WC = Fraction(0)
        else:
            WA = WB = Fraction(3 * 30)
            WC = Fraction(30)
    else:
        WA, WB, WC = (Fraction(v) for v in block_work(disc, level))
    tot = WA + 2 * WB + WC
    return WA / tot, WB / tot, WC / tot


def relaxation_work(disc, ahat, xi, level=None):
    wa, wb, wc = normalized_blocks(disc, level)
    w_ahat = wa if ahat == "f" else 2 * wa
    return xi * w_ahat + 2 * wb + wc


def fmg_work(disc, nu_pre, nu_post, nu_inc, kappa, ahat, xi, level=None):
    """W(FMG(s)) in WU (Eq. cost-var-fmg with Eq. bound-var-v-cycle)."""
    wp = relaxation_work(disc, ahat, xi, level)
    w_vll = (nu_pre + nu_post) * wp + 1
    w_star = Fraction(8, 7) * w_vll + Fraction(16, 49) * nu_inc * wp
    return Fraction(8 * kappa, 7) * w_star


def unknown_ratio_limit():
    """P2-P1 on level l over P1-P1 on level l+1 (Sec. 4.1): leading n^3
    coefficients of 3 (Nv + 6 No + Nx) + Nv over 4 N(2n)."""
    return Fraction(3 * (1 + 6 + 1) + 1, 4 * 8)
