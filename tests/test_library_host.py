"""Host-side checks of the C ABI library that need no GPU: it loads, exports
every entry point declared in include/hhg.h, validates macro meshes and
problem descriptions, and reports layouts and workspace sizes."""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

from hhg_inputs import cube24_macro_mesh, kuhn_box_macro_mesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hhg():
    from paper_2010_13513_gb300 import build, hhg as mod
    if not os.path.exists(mod.LIB_PATH):
        build.build()
    mod.load()
    return mod


def test_exports_every_declared_symbol(hhg):
    out = subprocess.run(["nm", "-D", "--defined-only", hhg.LIB_PATH], capture_output=True, text=True).stdout
    syms = {l.split()[-1] for l in out.splitlines() if l.strip()}
    declared = hhg.exported_symbols()
    assert len(declared) >= 20
    missing = [s for s in declared if s not in syms]
    assert not missing, missing


def _create(hhg, verts, tets):
    lib = hhg.load()
    v = np.ascontiguousarray(verts, dtype=np.float64)
    t = np.ascontiguousarray(tets, dtype=np.int32)
    h = C.c_void_p()
    rc = lib.hhg_mesh_create(v.ctypes.data_as(C.POINTER(C.c_double)), v.shape[0],
                             t.ctypes.data_as(C.POINTER(C.c_int)), t.shape[0], C.byref(h))
    if rc == 0:
        lib.hhg_mesh_destroy(h)
    return rc


@pytest.mark.parametrize("box", [(1, 1, 1), (2, 2, 2), (1, 2, 3)])
def test_mesh_accepts_kuhn_boxes(hhg, box):
    v, t = kuhn_box_macro_mesh(*box, H=0.5)
    assert _create(hhg, v, t) == 0


def test_mesh_rejects_other_meshes(hhg):
    v, t = kuhn_box_macro_mesh(1, 1, 1)
    assert _create(hhg, v, t[:5]) == -1                   # missing tetrahedron
    t2 = t.copy()
    t2[0] = [0, 1, 2, 4]                                    # corner simplex, not Kuhn
    assert _create(hhg, v, t2) == -1
    assert _create(hhg, v + 0.25, t) == -1                  # box not at the origin
    buf = C.create_string_buffer(256)
    hhg.load().hhg_last_error(buf, 256)
    assert b"origin" in buf.value
    # the paper's cube of 24 macro tetrahedra (corners, face centres, centre)
    # is not a Kuhn box: rejected with the reason
    v24, t24 = cube24_macro_mesh()
    assert _create(hhg, v24, t24) == -1
    hhg.load().hhg_last_error(buf, 256)
    assert b"Kuhn" in buf.value


def _problem(hhg, disc, L, lc, solve=0, err=0, box=(1, 1, 1), nu_a=0.0):
    lib = hhg.load()
    mesh = C.c_void_p()
    assert lib.hhg_mesh_create_box(*box, 1.0, C.byref(mesh)) == 0
    d = hhg.ProblemDesc(disc, L, lc, solve, nu_a, 1, err)
    pb = C.c_void_p()
    rc = lib.hhg_problem_create(mesh, C.byref(d), C.byref(pb))
    return rc, pb, mesh


def test_problem_layout_and_workspace(hhg):
    lib = hhg.load()
    rc, pb, mesh = _problem(hhg, hhg.P2P1, 3, 1, solve=1, err=1)
    assert rc == 0
    info = hhg.LayoutInfo()
    assert lib.hhg_layout(pb, 3, C.byref(info)) == 0
    assert (info.nx, info.groups) == (8, 8)
    assert info.n_velocity_nodes == 17 ** 3 and info.n_pressure_nodes == 9 ** 3
    assert info.n_dofs == 3 * 17 ** 3 + 9 ** 3
    assert info.vector_elems == 25 * info.array_elems and info.array_elems % 64 == 0
    assert lib.hhg_layout(pb, 4, C.byref(info)) == 0          # error level
    assert lib.hhg_layout(pb, 5, C.byref(info)) == -1
    nbytes = C.c_size_t()
    assert lib.hhg_problem_workspace_bytes(pb, C.byref(nbytes)) == 0
    assert nbytes.value > 0 and nbytes.value % 256 == 0
    # steps before binding a workspace are refused
    assert lib.hhg_apply(pb, 3, 0, 0, C.c_void_p(256), C.c_void_p(512)) == -7
    lib.hhg_problem_destroy(pb)
    lib.hhg_mesh_destroy(mesh)


def test_problem_rejects_bad_descriptions(hhg):
    assert _problem(hhg, 7, 3, 0)[0] == -1
    assert _problem(hhg, hhg.P1P1, 3, 4)[0] == -1
    assert _problem(hhg, hhg.P1P1, 3, 0, solve=5)[0] == -1


def test_bind_rejects_small_or_misaligned_workspace(hhg):
    lib = hhg.load()
    rc, pb, mesh = _problem(hhg, hhg.P1P1, 2, 0)
    assert rc == 0
    assert lib.hhg_problem_bind(pb, C.c_void_p(256), 16, None) == -2
    assert lib.hhg_problem_bind(pb, C.c_void_p(257), 1 << 40, None) == -1
    lib.hhg_problem_destroy(pb)
    lib.hhg_mesh_destroy(mesh)


def test_batch_and_host_solve_entry_points_reject_bad_arguments(hhg):
    """The batch and end-to-end entry points validate their arguments on the
    host before any device work: null handles and out-of-range groupings give
    HHG_EINVAL and an error text."""
    lib = hhg.load()
    EINVAL = -1
    assert lib.hhg_batch_create(None, 0, None) == EINVAL
    assert lib.hhg_batch_set_grouping(None, 0) == EINVAL
    assert lib.hhg_batch_get_grouping(None, None) == EINVAL
    a, b = C.c_int64(), C.c_int64()
    assert lib.hhg_batch_launch_counts(None, C.byref(a), C.byref(b)) == EINVAL
    prm = hhg.Params.make()
    assert lib.hhg_fmg_solve_host(None, C.byref(prm), None, None, None, None) == EINVAL
    buf = C.create_string_buffer(256)
    lib.hhg_last_error(buf, 256)
    assert buf.value


@pytest.mark.parametrize("disc", ["P1P1", "P2P1"])
def test_refinement_residual_kind_and_argument_checks(hhg, disc):
    """The refinement residual's arithmetic: double-float by default (constant
    and variable viscosity), FP64 on request; out-of-range kinds, null
    handles and unbound problems give errors before any device work."""
    lib = hhg.load()
    EINVAL, ESTATE = -1, -7
    d = hhg.P1P1 if disc == "P1P1" else hhg.P2P1
    kind = C.c_int(-1)
    rc, pb, mesh = _problem(hhg, d, 3, 1, solve=1)
    assert rc == 0
    assert lib.hhg_get_refinement_residual(pb, C.byref(kind)) == 0 and kind.value == hhg.REFINE["df32"]
    assert lib.hhg_set_refinement_residual(pb, hhg.REFINE["fp64"]) == 0
    assert lib.hhg_get_refinement_residual(pb, C.byref(kind)) == 0 and kind.value == hhg.REFINE["fp64"]
    assert lib.hhg_set_refinement_residual(pb, 7) == EINVAL
    assert lib.hhg_set_refinement_residual(pb, hhg.REFINE["df32"]) == 0
    assert lib.hhg_refinement_residual(pb, 3, C.c_void_p(256), C.c_void_p(256), C.c_void_p(256)) == ESTATE
    lib.hhg_problem_destroy(pb)
    lib.hhg_mesh_destroy(mesh)
    rc, pb, mesh = _problem(hhg, d, 3, 1, solve=1, nu_a=1.5)
    assert rc == 0
    assert lib.hhg_get_refinement_residual(pb, C.byref(kind)) == 0 and kind.value == hhg.REFINE["df32"]
    assert lib.hhg_set_refinement_residual(pb, hhg.REFINE["fp64"]) == 0
    assert lib.hhg_get_refinement_residual(pb, C.byref(kind)) == 0 and kind.value == hhg.REFINE["fp64"]
    assert lib.hhg_set_refinement_residual(pb, hhg.REFINE["df32"]) == 0
    lib.hhg_problem_destroy(pb)
    lib.hhg_mesh_destroy(mesh)
    assert lib.hhg_set_refinement_residual(None, 0) == EINVAL
    assert lib.hhg_get_refinement_residual(None, C.byref(kind)) == EINVAL
    assert lib.hhg_refinement_residual(None, 3, None, None, None) == EINVAL
