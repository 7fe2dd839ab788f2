"""Thin ctypes binding of libhhg.so (include/hhg.h).

Argument marshalling only: every step of the solve runs in the library's
CUDA kernels.  PyTorch provides the device memory (workspace and vectors)
and the CUDA stream.  There is no CPU fallback: loading fails loudly when
the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhhg.so")

P1P1 = 1
P2P1 = 2
FP64 = 0
FP32 = 1
SOLVE_FP64 = 0
SOLVE_MIXED = 1
OP = {"FULL": 0, "A": 1, "BT": 2, "B": 3, "C": 4, "MASS": 5}
REFINE = {"fp64": 0, "df32": 1}   # arithmetic of the refinement residual
AHAT = {"f": 0, "s": 1}


class ProblemDesc(C.Structure):
    _fields_ = [("disc", C.c_int), ("L", C.c_int), ("coarse_level", C.c_int), ("solve", C.c_int),
                ("nu_a", C.c_double), ("pspg_rhs", C.c_int), ("error_level", C.c_int),
                ("nn_hidden", C.c_int), ("nn_samples", C.c_int), ("nn_batch", C.c_int)]


class NNCfg(C.Structure):
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_double), ("n_train", C.c_int),
                ("seed", C.c_uint64), ("recorded", C.c_int), ("smooth_frac", C.c_double)]


class NNReport(C.Structure):
    _fields_ = [("n", C.c_int), ("n_params", C.c_int64), ("loss_first", C.c_double), ("loss_last", C.c_double),
                ("val_rel_err", C.c_double), ("train_ms", C.c_double)]


class LayoutInfo(C.Structure):
    _fields_ = [("level", C.c_int), ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("groups", C.c_int),
                ("sx", C.c_int), ("sy", C.c_int64), ("array_elems", C.c_int64), ("vector_elems", C.c_int64),
                ("n_velocity_nodes", C.c_int64), ("n_pressure_nodes", C.c_int64), ("n_dofs", C.c_int64),
                ("h", C.c_double)]


class Params(C.Structure):
    """The FMG tuple s = (nu_pre, nu_post, nu_inc, kappa, A_hat, xi) and omega^{-1}."""
    _fields_ = [("nu_pre", C.c_int), ("nu_post", C.c_int), ("nu_inc", C.c_int), ("kappa", C.c_int),
                ("ahat", C.c_int), ("xi", C.c_int), ("omega_inv", C.c_double)]

    @classmethod
    def make(cls, nu_pre=3, nu_post=3, nu_inc=0, kappa=1, ahat="s", xi=1, omega_inv=0.5):
        return cls(nu_pre, nu_post, nu_inc, kappa, AHAT[ahat] if isinstance(ahat, str) else ahat, xi, omega_inv)


class Stats(C.Structure):
    _fields_ = [("wu_model", C.c_double), ("wu_counted", C.c_double), ("res_u", C.c_double),
                ("res_p", C.c_double), ("kernel_launches", C.c_int64)]


_lib = None


def load():
    """Loads libhhg.so; raises if it is missing (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2010_13513_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P, VP, I, D, DP = C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.POINTER(C.c_double)
    sig = {
        "hhg_last_error": [C.c_char_p, C.c_size_t],
        "hhg_mesh_create": [DP, I, C.POINTER(C.c_int), I, C.POINTER(P)],
        "hhg_mesh_create_box": [I, I, I, D, C.POINTER(P)],
        "hhg_mesh_destroy": [P],
        "hhg_problem_create": [P, C.POINTER(ProblemDesc), C.POINTER(P)],
        "hhg_problem_workspace_bytes": [P, C.POINTER(C.c_size_t)],
        "hhg_problem_bind": [P, VP, C.c_size_t, VP],
        "hhg_problem_destroy": [P],
        "hhg_layout": [P, I, C.POINTER(LayoutInfo)],
        "hhg_vector_from_host": [P, I, I, DP, VP],
        "hhg_vector_to_host": [P, I, I, VP, DP],
        "hhg_set_rhs": [P, I, DP, DP],
        "hhg_set_rhs_levels": [P, I, I, C.POINTER(DP), C.POINTER(DP)],
        "hhg_level_vector": [P, I, I, C.POINTER(VP)],
        "hhg_apply": [P, I, I, I, VP, VP],
        "hhg_residual": [P, I, I, VP, VP, VP, DP],
        "hhg_refinement_residual": [P, I, VP, VP, VP],
        "hhg_set_refinement_residual": [P, I],
        "hhg_get_refinement_residual": [P, C.POINTER(C.c_int)],
        "hhg_smooth": [P, I, C.POINTER(Params), I, I, VP, VP],
        "hhg_restrict": [P, I, I, VP, VP],
        "hhg_prolongate_add": [P, I, I, VP, VP],
        "hhg_coarse_solve": [P, I, VP, VP],
        "hhg_vcycle": [P, I, C.POINTER(Params), I, VP, VP],
        "hhg_fmg_solve": [P, C.POINTER(Params), VP, C.POINTER(Stats)],
        "hhg_fmg_solve_host": [P, C.POINTER(Params), C.POINTER(DP), C.POINTER(DP), DP, C.POINTER(Stats)],
        "hhg_estimate_omega": [P, I, I, DP, DP],
        "hhg_set_graph_mode": [P, I],
        "hhg_set_small_level_mode": [P, I],
        "hhg_set_level_smoother": [P, I, I, I, I],
        "hhg_set_launch_shape": [P, I, I, I, I, I, I, I],
        "hhg_get_launch_shape": [P, I, C.POINTER(C.c_int)],
        "hhg_get_level_smoother": [P, I, I, C.POINTER(C.c_int), C.POINTER(C.c_int)],
        "hhg_set_level_sweep_order": [P, I, I],
        "hhg_get_level_sweep_order": [P, I, C.POINTER(C.c_int)],
        "hhg_error_norms": [P, I, VP, DP, DP, DP, DP],
        "hhg_block_norms_noalloc": [VP, I, C.c_int64, C.c_int64, VP, VP],
        "hhg_batch_create": [C.POINTER(P), I, C.POINTER(P)],
        "hhg_autotune": [P, I, C.POINTER(C.c_int)],
        "hhg_coarse_nn_size": [P, C.POINTER(C.c_int), C.POINTER(C.c_int64)],
        "hhg_coarse_nn_set_params": [P, C.POINTER(C.c_float)],
        "hhg_coarse_nn_get_params": [P, C.POINTER(C.c_float)],
        "hhg_coarse_nn_grad": [P, C.POINTER(C.c_float), C.POINTER(C.c_float), I, DP, C.POINTER(C.c_float)],
        "hhg_coarse_nn_train": [P, C.POINTER(NNCfg), C.POINTER(NNReport)],
        "hhg_coarse_nn_enable": [P, I, D],
        "hhg_coarse_nn_record": [P, I, C.POINTER(C.c_int64)],
        "hhg_coarse_nn_counts": [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
        "hhg_batch_destroy": [P],
        "hhg_batch_fmg_solve": [P, C.POINTER(Params), VP, C.POINTER(C.c_int64)],
        "hhg_batch_launch_counts": [P, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
        "hhg_batch_set_grouping": [P, I],
        "hhg_batch_get_grouping": [P, C.POINTER(C.c_int)],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = C.c_int
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C ABI entry points declared in include/hhg.h."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "hhg.h")
    with open(hdr) as f:
        return sorted(set(re.findall(r"^int (hhg_\w+)\(", f.read(), flags=re.M)))


class HHGError(RuntimeError):
    pass


def _host_ptr(a, n):
    """(double pointer, object keeping it alive) of n contiguous host doubles:
    a CPU float64 tensor is used in place, anything else through numpy."""
    if isinstance(a, torch.Tensor):
        if a.device.type != "cpu" or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() < n:
            raise ValueError("host tensor must be a contiguous CPU float64 tensor of the canonical length")
        return C.cast(a.data_ptr(), C.POINTER(C.c_double)), a
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.size < n:
        raise ValueError("host array shorter than the canonical length")
    return _dp(a), a


def _check(rc, what=""):
    if rc != 0:
        buf = C.create_string_buffer(1024)
        load().hhg_last_error(buf, 1024)
        raise HHGError(f"{what} failed ({rc}): {buf.value.decode()}")


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class Mesh:
    def __init__(self, handle):
        self.h = handle

    @classmethod
    def box(cls, mx, my, mz, H=1.0):
        lib = load()
        h = C.c_void_p()
        _check(lib.hhg_mesh_create_box(mx, my, mz, H, C.byref(h)), "hhg_mesh_create_box")
        return cls(h)

    @classmethod
    def from_tets(cls, verts, tets):
        lib = load()
        v = np.ascontiguousarray(verts, dtype=np.float64)
        t = np.ascontiguousarray(tets, dtype=np.int32)
        h = C.c_void_p()
        _check(lib.hhg_mesh_create(_dp(v), v.shape[0], t.ctypes.data_as(C.POINTER(C.c_int)), t.shape[0],
                                   C.byref(h)), "hhg_mesh_create")
        return cls(h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hhg_mesh_destroy(self.h)
            self.h = None


class Problem:
    """A level hierarchy coarse_level..L of one Stokes problem on one GPU."""

    def __init__(self, mesh: Mesh, disc="P1P1", L=4, coarse_level=0, solve="fp64", nu_a=0.0, pspg_rhs=True,
                 error_level=False, device="cuda", stream=None, nn_hidden=0, nn_samples=0, nn_batch=0):
        lib = load()
        self.disc = disc
        self.L, self.lc = L, coarse_level
        self.solve = solve
        d = ProblemDesc(P1P1 if disc == "P1P1" else P2P1, L, coarse_level,
                        SOLVE_MIXED if solve == "mixed" else SOLVE_FP64, float(nu_a), int(pspg_rhs), int(error_level),
                        int(nn_hidden), int(nn_samples), int(nn_batch))
        h = C.c_void_p()
        _check(lib.hhg_problem_create(mesh.h, C.byref(d), C.byref(h)), "hhg_problem_create")
        self.h = h
        self.mesh = mesh
        nbytes = C.c_size_t()
        _check(lib.hhg_problem_workspace_bytes(h, C.byref(nbytes)), "hhg_problem_workspace_bytes")
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        with torch.cuda.stream(self.stream):
            self.workspace = torch.empty(int(nbytes.value) + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        _check(lib.hhg_problem_bind(h, C.c_void_p(self._ws_ptr), nbytes.value, C.c_void_p(self.stream.cuda_stream)),
               "hhg_problem_bind")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hhg_problem_destroy(self.h)
            self.h = None

    # -------------------------------------------------------------- layout
    def layout(self, level):
        info = LayoutInfo()
        _check(load().hhg_layout(self.h, level, C.byref(info)), "hhg_layout")
        return info

    def new_vector(self, level, prec=FP64):
        n = self.layout(level).vector_elems
        with torch.cuda.stream(self.stream):
            return torch.zeros(n, dtype=torch.float64 if prec == FP64 else torch.float32, device=self.device)

    def to_device(self, level, host, prec=FP64, out=None):
        host = np.ascontiguousarray(host, dtype=np.float64)
        out = self.new_vector(level, prec) if out is None else out
        _check(load().hhg_vector_from_host(self.h, level, prec, _dp(host), _ptr(out)), "hhg_vector_from_host")
        return out

    def to_host(self, level, dev, prec=None, out=None):
        """Canonical FP64 host copy of a device vector; `out` may be a
        contiguous CPU float64 tensor (pinned memory: one fast copy)."""
        prec = (FP64 if dev.dtype == torch.float64 else FP32) if prec is None else prec
        info = self.layout(level)
        n = 3 * info.n_velocity_nodes + info.n_pressure_nodes
        host = np.zeros(n) if out is None else out
        ptr, host = _host_ptr(host, n)
        _check(load().hhg_vector_to_host(self.h, level, prec, _ptr(dev), ptr), "hhg_vector_to_host")
        return host

    def level_vector(self, level, which):
        """Library-owned FP64 vector as a torch view: 'rhs', 'W' or 'x'."""
        p = C.c_void_p()
        _check(load().hhg_level_vector(self.h, level, {"rhs": 0, "W": 1, "x": 2}[which], C.byref(p)),
               "hhg_level_vector")
        n = self.layout(level).vector_elems
        off = (p.value - self.workspace.data_ptr()) // 8
        assert (p.value - self.workspace.data_ptr()) % 8 == 0
        return self.workspace.view(torch.float64)[off:off + n] if (self.workspace.data_ptr() % 8 == 0) else None

    # ------------------------------------------------------------------ rhs
    def set_rhs(self, level, f_nodal, w_nodal):
        """Nodal forcing and Dirichlet data (3 x n_velocity_nodes each), numpy
        arrays or contiguous CPU float64 tensors (pinned memory: fast copies)."""
        n = 3 * self.layout(level).n_velocity_nodes
        fp, f = _host_ptr(f_nodal, n)
        wp, w = _host_ptr(w_nodal, n)
        _check(load().hhg_set_rhs(self.h, level, fp, wp), "hhg_set_rhs")

    def set_rhs_levels(self, l0, f_list, w_list):
        """set_rhs for levels l0 .. l0 + len(f_list) - 1 in one call (one
        synchronisation for all levels)."""
        n = len(f_list)
        if n == 0 or len(w_list) != n:
            raise ValueError("need one forcing and one Dirichlet array per level")
        dp = C.POINTER(C.c_double)
        keep, fps, wps = [], (dp * n)(), (dp * n)()
        for i in range(n):
            m = 3 * self.layout(l0 + i).n_velocity_nodes
            fp, f = _host_ptr(f_list[i], m)
            wp, w = _host_ptr(w_list[i], m)
            keep += [f, w]
            fps[i], wps[i] = fp, wp
        _check(load().hhg_set_rhs_levels(self.h, l0, l0 + n - 1, fps, wps), "hhg_set_rhs_levels")

    # ---------------------------------------------------------------- steps
    @staticmethod
    def _prec(t):
        return FP64 if t.dtype == torch.float64 else FP32

    def apply(self, level, op, x, y):
        _check(load().hhg_apply(self.h, level, OP[op], self._prec(x), _ptr(x), _ptr(y)), "hhg_apply")

    def residual(self, level, x, b, r, norms=False):
        nr = np.zeros(2)
        _check(load().hhg_residual(self.h, level, self._prec(x), _ptr(x), _ptr(b), _ptr(r),
                                   _dp(nr) if norms else None), "hhg_residual")
        return (float(nr[0]), float(nr[1])) if norms else None

    def refinement_residual(self, level, x, b, r):
        """r (FP32) = fl32(b - calA x) of the mixed solve's refinement step,
        x and b FP64 device tensors (hhg_refinement_residual)."""
        _check(load().hhg_refinement_residual(self.h, level, _ptr(x), _ptr(b), _ptr(r)), "hhg_refinement_residual")

    def set_refinement_residual(self, kind):
        """kind: "fp64" or "df32" (hhg_set_refinement_residual)."""
        _check(load().hhg_set_refinement_residual(self.h, REFINE[kind]), "hhg_set_refinement_residual")

    def refinement_residual_kind(self):
        k = C.c_int()
        _check(load().hhg_get_refinement_residual(self.h, C.byref(k)), "hhg_get_refinement_residual")
        return {v: n for n, v in REFINE.items()}[k.value]

    def smooth(self, level, prm, sweeps, x, b):
        _check(load().hhg_smooth(self.h, level, C.byref(prm), sweeps, self._prec(x), _ptr(x), _ptr(b)),
               "hhg_smooth")

    def restrict(self, level, rf, rc):
        _check(load().hhg_restrict(self.h, level, self._prec(rf), _ptr(rf), _ptr(rc)), "hhg_restrict")

    def prolongate_add(self, level, xc, xf):
        _check(load().hhg_prolongate_add(self.h, level, self._prec(xc), _ptr(xc), _ptr(xf)), "hhg_prolongate_add")

    def coarse_solve(self, b, x):
        _check(load().hhg_coarse_solve(self.h, self._prec(b), _ptr(b), _ptr(x)), "hhg_coarse_solve")

    def vcycle(self, level, prm, x, b):
        _check(load().hhg_vcycle(self.h, level, C.byref(prm), self._prec(x), _ptr(x), _ptr(b)), "hhg_vcycle")

    def fmg_solve(self, prm, x_out=None, stats=True):
        st = Stats()
        _check(load().hhg_fmg_solve(self.h, C.byref(prm), _ptr(x_out), C.byref(st) if stats else None),
               "hhg_fmg_solve")
        return st if stats else None

    def fmg_solve_host(self, prm, f_levels, w_levels, out=None, stats=True):
        """End-to-end solve from host nodal data of every level (coarse level
        first; CPU float64 tensors or arrays in canonical order, pinned memory
        for asynchronous copies); the solution in canonical order goes to
        `out` (a contiguous CPU float64 tensor or array of n_dofs, or None)."""
        n = self.L - self.lc + 1
        if len(f_levels) != n or len(w_levels) != n:
            raise ValueError("one f and one w per level from the coarse level to L")
        keep = []
        fp = (C.POINTER(C.c_double) * n)()
        wp = (C.POINTER(C.c_double) * n)()
        for i in range(n):
            nv = 3 * self.layout(self.lc + i).n_velocity_nodes
            fp[i], kf = _host_ptr(f_levels[i], nv)
            wp[i], kw = _host_ptr(w_levels[i], nv)
            keep += [kf, kw]
        xo = None
        if out is not None:
            xo, ko = _host_ptr(out, self.layout(self.L).n_dofs)
            keep.append(ko)
        st = Stats()
        _check(load().hhg_fmg_solve_host(self.h, C.byref(prm), fp, wp, xo, C.byref(st) if stats else None),
               "hhg_fmg_solve_host")
        return st if stats else None

    def set_graph_mode(self, on):
        _check(load().hhg_set_graph_mode(self.h, int(on)), "hhg_set_graph_mode")

    # ------------------------------------------- learned coarse correction
    def nn_size(self):
        n, p = C.c_int(), C.c_int64()
        _check(load().hhg_coarse_nn_size(self.h, C.byref(n), C.byref(p)), "hhg_coarse_nn_size")
        return n.value, p.value

    def nn_set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        _check(load().hhg_coarse_nn_set_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float))),
               "hhg_coarse_nn_set_params")

    def nn_get_params(self):
        _, p = self.nn_size()
        a = np.zeros(p, dtype=np.float32)
        _check(load().hhg_coarse_nn_get_params(self.h, a.ctypes.data_as(C.POINTER(C.c_float))),
               "hhg_coarse_nn_get_params")
        return a

    def nn_grad(self, X, T):
        X = np.ascontiguousarray(X, dtype=np.float32)
        T = np.ascontiguousarray(T, dtype=np.float32)
        _, p = self.nn_size()
        g = np.zeros(p, dtype=np.float32)
        loss = C.c_double()
        fp = C.POINTER(C.c_float)
        _check(load().hhg_coarse_nn_grad(self.h, X.ctypes.data_as(fp), T.ctypes.data_as(fp), X.shape[0],
                                         C.byref(loss), g.ctypes.data_as(fp)), "hhg_coarse_nn_grad")
        return loss.value, g

    def nn_train(self, epochs=30, batch=128, lr=1e-3, n_train=None, seed=2, smooth_frac=0.5, recorded=False):
        cfg = NNCfg(epochs, batch, lr, n_train, seed, int(recorded), smooth_frac)
        rep = NNReport()
        _check(load().hhg_coarse_nn_train(self.h, C.byref(cfg), C.byref(rep)), "hhg_coarse_nn_train")
        return rep

    def nn_record(self, on):
        c = C.c_int64()
        _check(load().hhg_coarse_nn_record(self.h, int(on), C.byref(c)), "hhg_coarse_nn_record")
        return c.value

    def nn_enable(self, mode, theta=0.1):
        _check(load().hhg_coarse_nn_enable(self.h, int(mode), float(theta)), "hhg_coarse_nn_enable")

    def nn_counts(self):
        a, r = C.c_int64(), C.c_int64()
        _check(load().hhg_coarse_nn_counts(self.h, C.byref(a), C.byref(r)), "hhg_coarse_nn_counts")
        return a.value, r.value

    def autotune(self, reps=5):
        """Per-level launch choices; returns {level: (row_threads,
        row_kplanes, gs_threads, resident_ctas, resident_threads,
        stream_threads, row_sites, gs_lanes, gs_lanes_vertex, bt_threads,
        bt_kplanes, bt_sites, bc_threads, bc_kplanes, bc_sites,
        gs_threads_vertex)}; stream_threads is the block size of the
        streaming kernel of the full operator (0: the plain kernels)."""
        n = self.L - self.lc + 1
        out = (C.c_int * (16 * n))()
        _check(load().hhg_autotune(self.h, reps, out), "hhg_autotune")
        return {self.lc + i: tuple(out[16 * i:16 * i + 16]) for i in range(n)}

    def set_launch_shape(self, level, row_threads, row_kplanes, gs_threads, row_tile=0, row_sites=1, gs_lanes=1):
        """row_tile: 0 = plain row kernels; 64/128/256 = the streaming kernels
        with that many threads per block (levels with nx >= 64), of 4 sites
        per thread, or 2 (FP32) with row_sites = 2."""
        _check(load().hhg_set_launch_shape(self.h, level, row_threads, row_kplanes, gs_threads, int(row_tile),
                                           int(row_sites), int(gs_lanes)), "hhg_set_launch_shape")

    def launch_shape(self, level):
        """(row_threads, row_kplanes, gs_threads, stream_threads, row_sites, gs_lanes) of a level;
        row_sites reads 2 when the streaming rows take 2 sites per thread."""
        out = (C.c_int * 6)()
        _check(load().hhg_get_launch_shape(self.h, level, out), "hhg_get_launch_shape")
        return tuple(out)

    def set_small_level_mode(self, on):
        _check(load().hhg_set_small_level_mode(self.h, int(on)), "hhg_set_small_level_mode")

    def _vprec(self):
        return FP32 if self.solve == "mixed" else FP64

    def set_level_smoother(self, level, ctas, threads=0, prec=None):
        """CTAs (0..16) and threads per CTA (0 = 1024) of the
        shared-memory-resident smoother of a level; ctas = 0: one launch per
        phase.  prec defaults to the V-cycle precision."""
        p = self._vprec() if prec is None else prec
        _check(load().hhg_set_level_smoother(self.h, level, p, ctas, threads), "hhg_set_level_smoother")

    def level_smoother(self, level, prec=None):
        """(ctas, threads) of the level's smoother."""
        p = self._vprec() if prec is None else prec
        c, t = C.c_int(), C.c_int()
        _check(load().hhg_get_level_smoother(self.h, level, p, C.byref(c), C.byref(t)), "hhg_get_level_smoother")
        return c.value, t.value

    def set_sweep_order(self, level, order):
        """0: every Gauss-Seidel phase on the three components; 1: component
        by component (same iterates)."""
        _check(load().hhg_set_level_sweep_order(self.h, level, int(order)), "hhg_set_level_sweep_order")

    def sweep_order(self, level):
        o = C.c_int()
        _check(load().hhg_get_level_sweep_order(self.h, level, C.byref(o)), "hhg_get_level_sweep_order")
        return o.value

    def estimate_omega(self, level, v0, iters=100):
        v = np.ascontiguousarray(v0, dtype=np.float64)
        out = C.c_double()
        _check(load().hhg_estimate_omega(self.h, level, iters, _dp(v), C.byref(out)), "hhg_estimate_omega")
        return out.value

    def error_norms(self, level, x, u_exact, p_exact):
        u = np.ascontiguousarray(u_exact, dtype=np.float64)
        p = np.ascontiguousarray(p_exact, dtype=np.float64)
        eu, ep = C.c_double(), C.c_double()
        _check(load().hhg_error_norms(self.h, level, _ptr(x), _dp(u), _dp(p), C.byref(eu), C.byref(ep)),
               "hhg_error_norms")
        return eu.value, ep.value


class Batch:
    """Independent problems solved by one CUDA graph of merged launches: each
    launch runs the same kernel for all problems whose sequences reach it,
    over the flat list of their work items."""

    def __init__(self, problems):
        lib = load()
        self.problems = list(problems)
        arr = (C.c_void_p * len(self.problems))(*[p.h.value for p in self.problems])
        h = C.c_void_p()
        _check(lib.hhg_batch_create(arr, len(self.problems), C.byref(h)), "hhg_batch_create")
        self.h = h

    def fmg_solve(self, params, stream=None):
        stream = stream if stream is not None else torch.cuda.current_stream()
        prm = (Params * len(params))(*params)
        k = C.c_int64()
        _check(load().hhg_batch_fmg_solve(self.h, prm, C.c_void_p(stream.cuda_stream), C.byref(k)),
               "hhg_batch_fmg_solve")
        return k.value

    def set_grouping(self, grouping):
        """0: cohorts of identical kernel sequences; 1: cohorts by structure
        only, whatever the sizes; 2: one graph branch per problem; -1
        (default): 0 when its cohorts hold four problems each on average,
        else 2."""
        _check(load().hhg_batch_set_grouping(self.h, int(grouping)), "hhg_batch_set_grouping")

    def grouping(self):
        """The grouping of the current graph (-1 before the first solve)."""
        g = C.c_int()
        _check(load().hhg_batch_get_grouping(self.h, C.byref(g)), "hhg_batch_get_grouping")
        return g.value

    def launch_counts(self):
        """(kernels of the batch graph, kernels of the problems' own sequences)."""
        a, b = C.c_int64(), C.c_int64()
        _check(load().hhg_batch_launch_counts(self.h, C.byref(a), C.byref(b)), "hhg_batch_launch_counts")
        return a.value, b.value

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hhg_batch_destroy(self.h)
            self.h = None


# --------------------------------------------------------------- helpers
def velocity_coords(info):
    """Canonical velocity node coordinates of a level (P1 lattice or doubled lattice)."""
    if info.groups == 1:
        n, hh = (info.nx + 1, info.ny + 1, info.nz + 1), info.h
    else:
        n, hh = (2 * info.nx + 1, 2 * info.ny + 1, 2 * info.nz + 1), info.h / 2
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1) * hh


def pressure_coords(info):
    k, j, i = np.meshgrid(np.arange(info.nz + 1), np.arange(info.ny + 1), np.arange(info.nx + 1), indexing="ij")
    return np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1) * info.h


def set_workload_rhs(pb: Problem, workload, levels=None):
    """Evaluates the workload's forcing and Dirichlet data at the nodes of
    every level and hands them to hhg_set_rhs (the assembly runs on the GPU)."""
    levels = range(pb.lc, pb.L + 1) if levels is None else levels
    for l in levels:
        info = pb.layout(l)
        X = velocity_coords(info)
        f = workload.forcing(X)
        w = workload.dirichlet(X)
        pb.set_rhs(l, f.T.ravel(), w.T.ravel())
