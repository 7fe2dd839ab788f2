"""Shared set-up for the GPU parity tests: the same seeded inputs for the
CUDA library (through its C ABI) and for the CPU oracle."""
import numpy as np

from hhg_inputs import Workload

OMEGA_INV = {"P1P1": 0.5, "P2P1": 0.3}


def lib_problem(box, L, disc, lc=0, solve="fp64", nu_a=0.0, error_level=False, workload=None, H=None):
    from paper_2010_13513_gb300 import hhg
    H = (1.0 / max(box)) if H is None else H
    mesh = hhg.Mesh.box(*box, H)
    pb = hhg.Problem(mesh, disc=disc, L=L, coarse_level=lc, solve=solve, nu_a=nu_a, error_level=error_level)
    if workload is not None:
        hhg.set_workload_rhs(pb, workload)
    return pb


def oracle_hierarchy(box, L, disc, lc=0, nu_a=0.0, workload=None, H=None):
    from oracle.stokes import StokesHierarchy
    H = (1.0 / max(box)) if H is None else H
    return StokesHierarchy(box, H, L, disc, coarse_level=lc, nu_a=nu_a, workload=workload)


def random_vector(lev, seed, zero_dirichlet=True):
    x = np.random.default_rng(seed).uniform(-1.0, 1.0, lev.size)
    if zero_dirichlet:
        x[:3 * lev.nv] *= np.tile(lev.vint, 3)
    return x


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def curl_workload(nu_a=0.0):
    return Workload("curl", nu_a=nu_a)
