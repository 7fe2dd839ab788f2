"""Benchmark: FMG-solved Stokes DoF/s at discretisation-error accuracy.

Workload (default): P2-P1 Taylor-Hood Stokes on the unit cube split into 6
macro tetrahedra, refined to level 7 (3 x 257^3 velocity + 129^3 pressure
DoFs = 53,070,468 incl. Dirichlet nodes), the paper's analytic cube solution
(Sec. 5.1.1), coarse level 2, one FMG solve per step with FP32 V-cycles
inside FP64 iterative refinement.  The inputs (right-hand sides of all
levels) are resident in HBM before the timed region; L2 is flushed before
every timed step (and the level-7 vectors are larger than L2) and each step
is timed alone with CUDA events on the solver's stream.

Also reported: the accuracy (gamma_u, gamma_p of Sec. 5.1: error against the
exact solution relative to the discretisation error) with the bound pair it
meets, the FP64-only GPU solve of the same workload, the learned coarse-grid
correction against the plain coarse solve, the operator-apply roofline on
level 7, the CPU oracle on a bounded sample on every host core and on one,
and an end-to-end number through the C ABI with host data.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {hhg,reference}]
                       [--workload {p2-l7,p2-l6,p1-visc,batched,tme,tme-disc}]
Multi-GPU: one independent replica per rank ("replicas only"), weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FMG-solved Stokes DoF/s at disc.-error accuracy; operator-apply HBM GB/s"
WORKLOADS = {
    "p2-l7": dict(disc="P2P1", box=(1, 1, 1), L=7, lc=2, kind="paper"),
    "p2-l6": dict(disc="P2P1", box=(1, 1, 1), L=6, lc=1, kind="paper"),
}
WORKLOAD = dict(WORKLOADS["p2-l7"])
# FMG tuple s = (nu_pre, nu_post, nu_inc, kappa, A_hat, xi): of the tuples of the
# search space S of Sec. 5.1 that reach (gamma_u, gamma_p) <= (2, 2) on level 7
# (`--workload tme-disc`), one of the two fastest on the GPU, with the widest
# accuracy margin (gamma_p ~ 1.03); omega^{-1} from 100 power iterations on
# the finest level
PARAMS = dict(nu_pre=1, nu_post=3, nu_inc=1, kappa=1, ahat="f", xi=3)
# tuples of the batched problems (levels 3..6): on these small levels one
# V-cycle per FMG level leaves the pressure short of discretisation accuracy
# (gamma_p 2-8 with the level-7 tuple above and (2,3,2,1,A_s,1), manufactured
# curl solution), two reach it: gamma below (1.01, 1.3) in the oracle at levels
# 3 and 4 for P2-P1, and (1.01, 0.95) at level 4 for P1-P1
BATCH_PARAMS = {"P1P1": dict(nu_pre=2, nu_post=2, nu_inc=2, kappa=2, ahat="s", xi=1),
                "P2P1": dict(nu_pre=1, nu_post=2, nu_inc=1, kappa=2, ahat="f", xi=3)}
# the accuracy bound (gamma_u, gamma_p) of a solve "at discretisation-error
# accuracy" (Sec. 5.1: both errors within a factor 2 of the discretisation
# error), and the bound pairs of Table 3 reported beside it
DISC_BOUND = (2.0, 2.0)
TABLE3_BOUNDS = [(1.1, 2.0), (1.1, 5.0), (2.0, 10.0)]
CPU_SAMPLE_LEVEL = 4


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
            return
        # the timed region starts only once the sampler is running (its first line is written)
        t0 = time.time()
        while time.time() - t0 < 10.0 and self.p.poll() is None:
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        rows = [l.strip().split(", ") for l in self.f.read().splitlines() if l.strip()]
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) >= 9 for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def make_problem(solve, error_level=False, nn=False):
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    w = WORKLOAD
    # the network's hidden width is well below the coarse system's size (1154)
    kw = dict(nn_hidden=128, nn_samples=10000, nn_batch=256) if nn else {}
    pb = hhg.Problem(hhg.Mesh.box(*w["box"], 1.0), disc=w["disc"], L=w["L"], coarse_level=w["lc"], solve=solve,
                     error_level=error_level, **kw)
    wl = Workload(w["kind"])
    hhg.set_workload_rhs(pb, wl)
    return pb, wl


def omega_inv(pb):
    info = pb.layout(WORKLOAD["L"])
    v0 = np.random.default_rng(0).uniform(-1, 1, info.n_pressure_nodes)
    return pb.estimate_omega(WORKLOAD["L"], v0, iters=100)


def accuracy(pb, wl, prm, x):
    """gamma_u, gamma_p (Eqs. error, gamma): error of the FMG result over the
    error of the discrete solution (residuals < 1e-12)."""
    import torch
    from paper_2010_13513_gb300 import hhg
    L = WORKLOAD["L"]
    info = pb.layout(L + 1)
    ue = wl.exact_velocity(hhg.velocity_coords(info)).T.ravel()
    pe = wl.exact_pressure(hhg.pressure_coords(info))
    e_fmg = pb.error_norms(L, x, ue, pe)
    xs = x.clone()
    b = pb.level_vector(L, "rhs")
    r = pb.new_vector(L)
    cycles = 0
    for cycles in range(1, 400):
        pb.vcycle(L, prm, xs, b)
        nu, npp = pb.residual(L, xs, b, r, norms=True)
        if max(nu, npp) < 1e-12:
            break
    e_disc = pb.error_norms(L, xs, ue, pe)
    torch.cuda.synchronize()
    return e_fmg[0] / e_disc[0], e_fmg[1] / e_disc[1], e_fmg, e_disc, cycles, (nu, npp)


def time_steps(pb, prm, x, steps, warmup, stream):
    import torch
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        pb.fmg_solve(prm, x, stats=False)
    torch.cuda.synchronize()
    times = []
    for _ in range(steps):
        flush.fill_(1.0)                          # evict L2 (512 MB > 129 MB)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        pb.fmg_solve(prm, x, stats=False)
        e.record(stream)
        e.synchronize()
        times.append(s.elapsed_time(e))
    return times


def apply_roofline(pb, steps=20):
    """Average duration of the FP32 operator apply y = calA x on the finest
    level, each launch timed alone after an L2 flush."""
    import torch
    L = WORKLOAD["L"]
    info = pb.layout(L)
    x = pb.new_vector(L, prec=1)
    x.uniform_(-1, 1)
    y = pb.new_vector(L, prec=1)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(3):
        pb.apply(L, "FULL", x, y)
    ts = []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(st)
        pb.apply(L, "FULL", x, y)
        e.record(st)
        e.synchronize()
        ts.append(s.elapsed_time(e))
    t = statistics.mean(ts) * 1e-3
    alg_bytes = info.n_dofs * 4 * 2           # read every DoF once, write every DoF once (FP32)
    return alg_bytes, t


def kernel_source_hash():
    """sha256 of the sources of the streaming stencil-row kernel (the apply
    kernel of the roofline line): its source and header, and the generator
    and stencil builder that produce its compile-time row structure."""
    import hashlib
    h = hashlib.sha256()
    for f in ("stream.cu", "stream.h", "gen_structure.cpp", "stencils.cpp"):
        path = os.path.join(ROOT, "paper_2010_13513_gb300", "csrc", f)
        if os.path.exists(path):
            with open(path, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()


TRAFFIC_PROFILE = "profiles/apply_{disc}_l{L}_fp32.md"


def measured_traffic(shape):
    """DRAM bytes per launch of the roofline apply from the committed ncu
    summary of that kernel and workload, if it was taken on the current
    kernel sources with the same apply launch shape -- streaming-row threads
    per CTA and sites per thread, slots 3 and 4 of the level's launch shape --
    (else None)."""
    path = os.path.join(ROOT, TRAFFIC_PROFILE.format(disc=WORKLOAD["disc"].lower(), L=WORKLOAD["L"]))
    try:
        fields = dict(l.strip("- \n").split(": ", 1) for l in open(path) if l.startswith("- ") and ": " in l)
        if fields.get("kernel_source_sha256") == kernel_source_hash() and \
                fields.get("apply_shape") == json.dumps([shape[3], shape[4]]):
            return int(fields["dram_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def profile_apply(workload):
    """Only the roofline apply: set-up, three warm-up launches, then three
    launches (each after an L2 flush) between cudaProfilerStart/Stop.  The
    default workload's level-7 P2-P1 FP32 apply, or (p1-visc) the level-7
    P1-P1 FP32 apply on the 48-tetrahedron cube with nu = exp(a z)."""
    import torch
    from hhg_inputs import draw_viscosity_exponent
    from paper_2010_13513_gb300 import hhg
    torch.cuda.set_stream(torch.cuda.Stream())
    if workload == "p1-visc":
        L = 7
        pb = hhg.Problem(hhg.Mesh.box(2, 2, 2, 0.5), disc="P1P1", L=L, coarse_level=0, solve="mixed",
                         nu_a=draw_viscosity_exponent(0))
    else:
        L = WORKLOAD["L"]
        pb, _ = make_problem("mixed")
    pb.autotune(reps=3)
    x = pb.new_vector(L, prec=1)
    x.uniform_(-1, 1)
    y = pb.new_vector(L, prec=1)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(3):
        pb.apply(L, "FULL", x, y)
    torch.cuda.synchronize()
    print("launch shape", pb.launch_shape(L))
    torch.cuda.profiler.start()
    for _ in range(3):
        flush.fill_(1.0)
        pb.apply(L, "FULL", x, y)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()


def e2e_steps(pb, wl, prm, steps, profile=False):
    """Through the public API with host data (hhg_fmg_solve_host): nodal
    forcing/Dirichlet data of every level from pinned host memory, assembled
    on the GPU (the finest level beside the FMG stages below it), the FMG
    solve, and the solution copied back to the host."""
    import torch
    from paper_2010_13513_gb300 import hhg
    L = WORKLOAD["L"]
    host = {}
    h2d = 0
    for l in range(WORKLOAD["lc"], L + 1):       # the step's inputs, in pinned host memory
        info = pb.layout(l)
        X = hhg.velocity_coords(info)
        f = torch.from_numpy(np.ascontiguousarray(wl.forcing(X).T.ravel())).pin_memory()
        w = torch.from_numpy(np.ascontiguousarray(wl.dirichlet(X).T.ravel())).pin_memory()
        host[l] = (f, w)
        h2d += 8 * (f.numel() + w.numel())
    d2h = pb.layout(L).n_dofs * 8
    out = torch.empty(pb.layout(L).n_dofs, dtype=torch.float64).pin_memory()

    fl = [host[l][0] for l in sorted(host)]
    wl_ = [host[l][1] for l in sorted(host)]

    def step():
        pb.fmg_solve_host(prm, fl, wl_, out=out, stats=False)

    step()                                       # warm-up (not timed)
    if profile:
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return [], h2d, d2h
    ts = []
    for _ in range(steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step()
        ts.append(time.perf_counter() - t0)
    assert torch.isfinite(out).all()
    return ts, h2d, d2h


def _host_cpu():
    """(usable cores, CPU model) of the host."""
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    model = ""
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu part", "hardware") and ":" in line:
                model = line.split(":", 1)[1].strip()
                if key == "model name":
                    break
    except OSError:
        pass
    import platform
    return cores, f"{platform.machine()} {model}".strip()


_ORACLE = {}


def _oracle_init(w, level, prm_dict):
    """Pool initialiser: the oracle's hierarchy of the sample (assembly is
    set-up, not timed) and one untimed solve."""
    from hhg_inputs import Workload
    from oracle.stokes import Params, StokesHierarchy
    hy = StokesHierarchy(w["box"], 1.0, level, w["disc"], coarse_level=min(w["lc"], level),
                         workload=Workload(w["kind"]))
    prm = Params(**prm_dict)
    hy.fmg(prm)
    _ORACLE.update(hy=hy, prm=prm, dofs=hy.lv[level].size)


def _oracle_fmg(_):
    t0 = time.perf_counter()
    _ORACLE["hy"].fmg(_ORACLE["prm"])
    return time.perf_counter() - t0, _ORACLE["dofs"]


def _oracle_pool(n, prm_dict, level):
    """n spawned single-threaded processes, each holding the oracle's
    hierarchy of the level-`level` sample of the workload (spawn: safe after
    CUDA initialisation; BLAS threads pinned to one per process)."""
    import multiprocessing as mp
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    return mp.get_context("spawn").Pool(n, initializer=_oracle_init, initargs=(dict(WORKLOAD), level, prm_dict))


def cpu_baseline(prm_dict, level=CPU_SAMPLE_LEVEL, seconds=10.0):
    """The FP64 CPU oracle as it stands: FMG on the same workload at a smaller
    level (bounded sample), on every host core (one independent solve per
    core at a time, single-threaded processes) and on one core."""
    cores, model = _host_cpu()
    out = {}
    for n in (cores, 1):
        with _oracle_pool(n, prm_dict, level) as pool:
            pool.map(_oracle_fmg, range(n))               # every worker warm
            t0 = time.perf_counter()
            solves, dofs = 0, 0
            while time.perf_counter() - t0 < seconds / 2:
                res = pool.map(_oracle_fmg, range(n))
                solves += len(res)
                dofs = res[0][1]
            dt = time.perf_counter() - t0
        out[n] = (solves * dofs / dt, solves, dt, dofs)
    v, solves, dt, dofs = out[cores]
    return {"value": v, "unit": "DoF/s", "cores": cores, "kind": "oracle",
            "sample": f"{WORKLOAD['disc']} 6-tet cube level {level} ({dofs} DoF), {solves} FMG solves in {dt:.1f} s on "
                      f"{cores} single-threaded processes (numpy/scipy oracle), host {model}",
            "single_core": {"value": out[1][0], "unit": "DoF/s", "cores": 1, "solves": out[1][1]}}


def aligned_batch(timed, n=48, L=4):
    """A batch whose kernel sequences align op for op: n P2-P1 problems on the
    unit cube at level L (random smooth forcing, one seed each), merged
    (grouping 0) against one graph branch per problem (grouping 2) and the
    same solves one after another."""
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    pbs, prms = [], []
    for i in range(n):
        pb = hhg.Problem(hhg.Mesh.box(1, 1, 1, 1.0), disc="P2P1", L=L, coarse_level=1, solve="mixed")
        hhg.set_workload_rhs(pb, Workload("modes", seed=9000 + i, box=(1, 1, 1), H=1.0))
        pbs.append(pb)
        prms.append(hhg.Params.make(**dict(BATCH_PARAMS["P2P1"], omega_inv=0.32)))
    pbs[0].autotune(reps=2)
    batch = hhg.Batch(pbs)
    out = {"problems": n, "workload": f"P2-P1 unit cube level {L}", "dofs": pbs[0].layout(L).n_dofs * n}
    batch.fmg_solve(prms)
    out["grouping_used"] = batch.grouping()
    for grouping in (0, 2):
        batch.set_grouping(grouping)
        batch.fmg_solve(prms)
        out[f"grouping_{grouping}"] = {"ms": timed(lambda: batch.fmg_solve(prms), 10) * 1e3,
                                      "graph_kernels": batch.launch_counts()[0]}
    out["sequential_ms"] = timed(lambda: [pb.fmg_solve(prm, None, stats=False) for pb, prm in zip(pbs, prms)], 3) * 1e3
    return out


def accuracy_batch(n=24, levels=(3, 5)):
    """Accuracy of batched solves at discretisation-error level: n uneven
    problems (Kuhn boxes {1,2}^3, levels 3..5, P1-P1 / P2-P1) with the
    manufactured curl solution, solved together by one batch graph; gamma_u,
    gamma_p (Eq. gamma) of every problem, the largest of each, and whether all
    meet the (2, 2) bound and the Table 3 bound pairs."""
    import torch
    from hhg_inputs import Workload, batched_problem_list
    from paper_2010_13513_gb300 import hhg
    specs = batched_problem_list(1, n=n, levels=levels)
    pbs, prms, wls = [], [], []
    for sp in specs:
        lc = 0 if sp["disc"] == "P1P1" else 1
        H = 1.0 / max(sp["box"])
        pb = hhg.Problem(hhg.Mesh.box(*sp["box"], H), disc=sp["disc"], L=sp["level"], coarse_level=lc, solve="mixed",
                         error_level=True)
        wl = Workload("curl", box=sp["box"], H=H)
        hhg.set_workload_rhs(pb, wl)
        info = pb.layout(sp["level"])
        om = pb.estimate_omega(sp["level"], np.random.default_rng(sp["seed"]).uniform(-1, 1, info.n_pressure_nodes), 30)
        s = BATCH_PARAMS[sp["disc"]]
        prms.append(hhg.Params.make(**s, omega_inv=om))
        pbs.append(pb)
        wls.append(wl)
    batch = hhg.Batch(pbs)
    batch.fmg_solve(prms)
    torch.cuda.synchronize()
    rows = []
    for sp, pb, prm, wl in zip(specs, pbs, prms, wls):
        L = sp["level"]
        gu, gp = _gamma(pb, wl, prm, pb.level_vector(L, "x").clone(), L)
        rows.append({"disc": sp["disc"], "box": list(sp["box"]), "level": L, "gamma_u": gu, "gamma_p": gp})
    gu_max = max(r["gamma_u"] for r in rows)
    gp_max = max(r["gamma_p"] for r in rows)
    return {"workload": f"{n} problems, Kuhn boxes {{1,2}}^3, levels {levels[0]}..{levels[1]}, P1-P1 / P2-P1, "
                        "manufactured curl solution, one batch graph",
            "grouping_used": batch.grouping(), "gamma_u_max": gu_max, "gamma_p_max": gp_max,
            "all_within": {f"({bu}, {bp})": all(r["gamma_u"] <= bu and r["gamma_p"] <= bp for r in rows)
                           for bu, bp in ((2, 2), (1.1, 2), (1.1, 5), (2, 10))},
            "problems": rows}


def run_batched(args):
    """The batched workload: 64 independent problems (Kuhn boxes {1,2}^3,
    levels 3..6, P1-P1 / P2-P1, random smooth forcing, zero Dirichlet data)
    solved by one CUDA graph of merged launches (each launch runs one kernel
    over the work items of all problems that reach it), against the same
    problems solved one after another (each with its own graph)."""
    import torch
    from hhg_inputs import Workload, batched_problem_list
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    specs = batched_problem_list(0)
    pbs, prms, dofs = [], [], 0
    t_setup = time.perf_counter()
    for sp in specs:
        lc = 0 if sp["disc"] == "P1P1" else 1
        H = 1.0 / max(sp["box"])
        pb = hhg.Problem(hhg.Mesh.box(*sp["box"], H), disc=sp["disc"], L=sp["level"], coarse_level=lc, solve="mixed")
        hhg.set_workload_rhs(pb, Workload("modes", seed=sp["seed"], box=sp["box"], H=H))
        pb.autotune(reps=2)
        info = pb.layout(sp["level"])
        om = pb.estimate_omega(sp["level"], np.random.default_rng(sp["seed"]).uniform(-1, 1, info.n_pressure_nodes), 30)
        s = BATCH_PARAMS[sp["disc"]]
        prms.append(hhg.Params.make(**s, omega_inv=om))
        pbs.append(pb)
        dofs += info.n_dofs
    t_setup = time.perf_counter() - t_setup
    batch = hhg.Batch(pbs)
    kernels = batch.fmg_solve(prms, stream)
    for pb, prm in zip(pbs, prms):
        pb.fmg_solve(prm, None, stats=False)
    torch.cuda.synchronize()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for _ in range(reps):
            fn()
        e.record(stream)
        e.synchronize()
        return s.elapsed_time(e) / reps * 1e-3

    sampler = ClockSampler(0)
    graph_kernels, problem_kernels = batch.launch_counts()
    t_batch = timed(lambda: batch.fmg_solve(prms, stream), args.steps)
    t_seq = timed(lambda: [pb.fmg_solve(prm, None, stats=False) for pb, prm in zip(pbs, prms)], max(1, args.steps // 2))
    # the other groupings of the batch's sequences (hhg_batch_set_grouping)
    used = batch.grouping()
    groupings = {used: {"ms": t_batch * 1e3, "graph_kernels": graph_kernels}}
    for grouping in (0, 1, 2):
        if grouping == used:
            continue
        batch.set_grouping(grouping)
        batch.fmg_solve(prms, stream)
        groupings[grouping] = {"ms": timed(lambda: batch.fmg_solve(prms, stream), args.steps) * 1e3,
                               "graph_kernels": batch.launch_counts()[0]}
    batch.set_grouping(-1)
    aligned = aligned_batch(timed)
    clocks = sampler.stop()
    gamma_batch = accuracy_batch()
    # accuracy of a few problems: delta against the discrete solution (Eq. relative-error)
    deltas = []
    for idx in (0, 1, 2):
        pb, prm = pbs[idx], prms[idx]
        L = pb.L
        x = pb.level_vector(L, "x").clone()
        xs = x.clone()
        b = pb.level_vector(L, "rhs")
        r = pb.new_vector(L)
        for _ in range(300):
            pb.vcycle(L, prm, xs, b)
            if max(pb.residual(L, xs, b, r, norms=True)) < 1e-12:
                break
        info = pb.layout(L)
        po = 3 * info.groups * info.array_elems
        du = float(torch.linalg.norm(x[:po] - xs[:po]) / torch.linalg.norm(xs[:po]))
        dp = float(torch.linalg.norm(x[po:] - xs[po:]) / torch.linalg.norm(xs[po:]))
        deltas.append({"problem": idx, "disc": specs[idx]["disc"], "level": specs[idx]["level"], "delta_u": du,
                       "delta_p": dp})
    line = {"metric": "batched FMG-solved Stokes DoF/s", "value": dofs / t_batch, "unit": "DoF/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": "64 independent Stokes problems: Kuhn boxes {1,2}^3, levels 3..6, P1-P1 and P2-P1, "
                                   "random smooth forcing (8 sine modes per component), zero Dirichlet data",
                       "dofs": dofs, "problems": len(pbs), "params": BATCH_PARAMS, "graph_kernels": graph_kernels,
                       "problem_kernels": problem_kernels, "setup_s": t_setup,
                       "grouping_used": used,
                       "groupings": {"0 (cohorts of identical sequences)": groupings[0],
                                     "1 (cohorts by structure)": groupings[1],
                                     "2 (one branch per problem, no merging)": groupings[2]},
                       "sequential_ms": t_seq * 1e3, "batch_speedup_vs_sequential": t_seq / t_batch,
                       "aligned_batch": aligned,
                       "accuracy": deltas, "accuracy_gamma": gamma_batch},
            "clocks": clocks}
    print(json.dumps(line))


def _gamma(pb, wl, prm, x, L, max_cycles=300):
    """gamma_u, gamma_p of Eq. gamma for the FP64 solution x of level L."""
    import torch
    from paper_2010_13513_gb300 import hhg
    info = pb.layout(L + 1)
    ue = wl.exact_velocity(hhg.velocity_coords(info)).T.ravel()
    pe = wl.exact_pressure(hhg.pressure_coords(info))
    e_fmg = pb.error_norms(L, x, ue, pe)
    xs = x.clone()
    b = pb.level_vector(L, "rhs")
    r = pb.new_vector(L)
    for _ in range(max_cycles):
        pb.vcycle(L, prm, xs, b)
        if max(pb.residual(L, xs, b, r, norms=True)) < 1e-12:
            break
    e_disc = pb.error_norms(L, xs, ue, pe)
    torch.cuda.synchronize()
    return e_fmg[0] / e_disc[0], e_fmg[1] / e_disc[1]


def _timed(fn, steps, warmup, stream):
    import torch
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    for _ in range(warmup):
        fn()
    ts = []
    for _ in range(steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        e.synchronize()
        ts.append(s.elapsed_time(e) * 1e-3)
    return statistics.mean(ts)


def run_p1_visc(args):
    """P1-P1 PSPG, 48-tetrahedron cube (2x2x2 Kuhn box on [0,1]^3) on level 7,
    viscosity nu = exp(a z) with a ~ U[0,4] from seed 0, FP32 V-cycles inside
    FP64 iterative refinement; Table 3 tuple (2,3,2,1,A_s,1)."""
    import torch
    from hhg_inputs import Workload, draw_viscosity_exponent
    from paper_2010_13513_gb300 import hhg
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    a = draw_viscosity_exponent(0)
    L = 7
    wl = Workload("curl", nu_a=a)
    pb = hhg.Problem(hhg.Mesh.box(2, 2, 2, 0.5), disc="P1P1", L=L, coarse_level=0, solve="mixed", nu_a=a,
                     error_level=True)
    hhg.set_workload_rhs(pb, wl)
    shapes = pb.autotune(reps=3)
    info = pb.layout(L)
    om = pb.estimate_omega(L, np.random.default_rng(0).uniform(-1, 1, info.n_pressure_nodes), 100)
    prm = hhg.Params.make(2, 3, 2, 1, "s", 1, om)
    x = pb.new_vector(L)
    st = pb.fmg_solve(prm, x)
    sampler = ClockSampler(0)
    t = _timed(lambda: pb.fmg_solve(prm, x, stats=False), args.steps, args.warmup, stream)
    clocks = sampler.stop()
    gu, gp = _gamma(pb, wl, prm, x, L)
    # the same solve with the FP64 refinement defect instead of the double-float one
    refine = {"kind": pb.refinement_residual_kind()}
    if refine["kind"] == "df32":
        xf = pb.new_vector(L)
        pb.set_refinement_residual("fp64")
        tf = _timed(lambda: pb.fmg_solve(prm, xf, stats=False), max(3, args.steps // 2), 2, stream)
        pb.set_refinement_residual("df32")
        refine.update({"fp64_refinement_ms_per_step": tf * 1e3, "df32_speedup": tf / t,
                       "rel_diff_vs_fp64_refinement": float(torch.linalg.norm(x - xf) / torch.linalg.norm(xf))})
        del xf
    # operator apply roofline at this size (FP32)
    xa = pb.new_vector(L, 1)
    xa.uniform_(-1, 1)
    ya = pb.new_vector(L, 1)
    ta = _timed(lambda: pb.apply(L, "FULL", xa, ya), 10, 3, stream)
    pk, src = peaks()
    ach = info.n_dofs * 8 / ta / 1e9
    print(json.dumps({
        "metric": "FMG-solved Stokes DoF/s at disc.-error accuracy", "value": info.n_dofs / t, "unit": "DoF/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"P1-P1 PSPG, 48-tet cube, level 7, nu = exp({a:.4f} z), curl solution, FP32 V-cycles "
                               "in FP64 refinement", "dofs": info.n_dofs, "omega_inv": om,
                   "params": [2, 3, 2, 1, "s", 1], "gamma_u": gu, "gamma_p": gp, "wu_model": st.wu_model,
                   "refinement_residual": refine,
                   "launch_shapes": {str(k): v for k, v in shapes.items()}},
        "roofline": {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": ach / pk["hbm_gbs"], "kernel": "FP32 FULL apply, level 7", "avg_launch_us": ta * 1e6,
                     "peak_source": src},
        "clocks": clocks}))


def run_tme(args):
    """The paper's parameter study (Sec. 5.1, Table 3) on the GPU: for P1-P1
    at level 6 and P2-P1 at level 5 on the 6-tetrahedron cube with the cube
    solution of Sec. 5.1.1, omega^{-1} by 100 power iterations, then one FMG
    solve for every tuple of the search space S,
    gamma_u and gamma_p against the discrete solution's error (Eq. gamma), the
    model work W(FMG(s)), and the minimal-work tuple under the three bound
    pairs of Table 3 (kappa = 1, as there, and with kappa = 2 allowed: all 768
    tuples of S).  (The paper's mesh has 24 macro tetrahedra; the study and
    the work model are the same.)"""
    import itertools
    import torch
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    torch.cuda.set_stream(torch.cuda.Stream())
    bounds = [(1.1, 2.0), (1.1, 5.0), (2.0, 10.0)]
    pairs = [("f", 1), ("f", 2), ("f", 3), ("f", 4), ("s", 1), ("s", 2)]
    out = {}
    t0 = time.perf_counter()
    for disc, L, lc in (("P1P1", 6, 0), ("P2P1", 5, 1)):
        wl = Workload("paper")
        pb = hhg.Problem(hhg.Mesh.box(1, 1, 1, 1.0), disc=disc, L=L, coarse_level=lc, solve="fp64", error_level=True)
        hhg.set_workload_rhs(pb, wl)
        pb.set_graph_mode(False)                 # one solve per tuple: no graph per tuple
        info = pb.layout(L)
        om = pb.estimate_omega(L, np.random.default_rng(0).uniform(-1, 1, info.n_pressure_nodes), 100)
        fine = pb.layout(L + 1)
        ue = wl.exact_velocity(hhg.velocity_coords(fine)).T.ravel()
        pe = wl.exact_pressure(hhg.pressure_coords(fine))
        # the discrete solution's error (residuals below 1e-12)
        prm0 = hhg.Params.make(3, 3, 0, 1, "s", 2, om)
        xs = pb.new_vector(L)
        b = pb.level_vector(L, "rhs")
        r = pb.new_vector(L)
        for _ in range(300):
            pb.vcycle(L, prm0, xs, b)
            if max(pb.residual(L, xs, b, r, norms=True)) < 1e-12:
                break
        e_disc = pb.error_norms(L, xs, ue, pe)
        rows = []
        x = pb.new_vector(L)
        for kap, npre, npost, ninc, (ah, xi) in itertools.product((1, 2), range(4), range(4), range(4), pairs):
            prm = hhg.Params.make(npre, npost, ninc, kap, ah, xi, om)
            st = pb.fmg_solve(prm, x)
            eu, ep = pb.error_norms(L, x, ue, pe)
            rows.append({"s": [npre, npost, ninc, kap, ah, xi], "wu": st.wu_model,
                         "gamma_u": eu / e_disc[0], "gamma_p": ep / e_disc[1]})

        def minimal(cands):
            best = []
            for gu, gp in bounds:
                ok = [q for q in cands if q["gamma_u"] <= gu and q["gamma_p"] <= gp]
                q = min(ok, key=lambda q: q["wu"]) if ok else None
                best.append({"bounds": [gu, gp], **(q or {"s": None})})
            return best

        k1 = [q for q in rows if q["s"][3] == 1]
        out[f"{disc}_L{L}"] = {"dofs": info.n_dofs, "omega_inv": om, "err_disc": e_disc, "tuples": len(rows),
                               "solved_gamma_le_2": sum(q["gamma_u"] <= 2 and q["gamma_p"] <= 2 for q in k1),
                               "min_gamma_p": min(q["gamma_p"] for q in rows), "table3": minimal(k1),
                               "kappa_le_2": minimal(rows)}
        del pb
    dt = time.perf_counter() - t0
    print(json.dumps({"metric": "TME parameter study (Table 3): minimal W(FMG(s)) under gamma bounds",
                      "value": dt, "unit": "s (whole study)", "n_gpus": 1, "higher_is_better": False,
                      "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "6-tet cube, cube solution of Sec. 5.1.1, the search space S "
                                             "(2 x 4 x 4 x 4 x 6 = 768 tuples per discretisation), FP64 solves",
                                 "results": out}}))


def run_tme_disc(args):
    """The work needed for discretisation-error accuracy at the benchmark's
    sizes: P2-P1 on the 6-tetrahedron cube at levels 6 and 7 (coarse level
    2, the paper's cube solution, FP32 V-cycles in FP64 refinement, omega^{-1}
    by 100 power iterations), one FMG solve for every tuple of the search
    space S of Sec. 5.1, gamma_u and gamma_p against the discrete solution's
    error (Eq. gamma), the model work W(FMG(s)), and the minimal-work tuple
    under the disc.-accuracy bound (2, 2) and the Table 3 bound pairs."""
    import itertools
    import torch
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    torch.cuda.set_stream(torch.cuda.Stream())
    bounds = [DISC_BOUND] + TABLE3_BOUNDS
    pairs = [("f", 1), ("f", 2), ("f", 3), ("f", 4), ("s", 1), ("s", 2)]
    out = {}
    t0 = time.perf_counter()
    for L in (6, 7):
        wl = Workload("paper")
        pb = hhg.Problem(hhg.Mesh.box(1, 1, 1, 1.0), disc="P2P1", L=L, coarse_level=2, solve="mixed",
                         error_level=True)
        hhg.set_workload_rhs(pb, wl)
        pb.autotune(reps=2)
        info = pb.layout(L)
        om = pb.estimate_omega(L, np.random.default_rng(0).uniform(-1, 1, info.n_pressure_nodes), 100)
        fine = pb.layout(L + 1)
        ue = wl.exact_velocity(hhg.velocity_coords(fine)).T.ravel()
        pe = wl.exact_pressure(hhg.pressure_coords(fine))
        prm0 = hhg.Params.make(3, 3, 0, 1, "s", 2, om)
        xs = pb.new_vector(L)
        b = pb.level_vector(L, "rhs")
        r = pb.new_vector(L)
        for _ in range(300):
            pb.vcycle(L, prm0, xs, b)
            if max(pb.residual(L, xs, b, r, norms=True)) < 1e-12:
                break
        e_disc = pb.error_norms(L, xs, ue, pe)
        del xs, r
        rows = []
        x = pb.new_vector(L)
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        for kap, npre, npost, ninc, (ah, xi) in itertools.product((1, 2), range(4), range(4), range(4), pairs):
            prm = hhg.Params.make(npre, npost, ninc, kap, ah, xi, om)
            st = pb.fmg_solve(prm, x)            # records this tuple's graph
            eu, ep = pb.error_norms(L, x, ue, pe)
            s0.record(pb.stream)
            pb.fmg_solve(prm, x, stats=False)    # graph replay, timed
            s1.record(pb.stream)
            s1.synchronize()
            rows.append({"s": [npre, npost, ninc, kap, ah, xi], "wu": st.wu_model, "ms": s0.elapsed_time(s1),
                         "gamma_u": eu / e_disc[0], "gamma_p": ep / e_disc[1]})
        pb.set_graph_mode(False)                 # frees the tuples' graphs
        best, fastest, best_k1 = [], [], []
        for gu, gp in bounds:
            ok = [q for q in rows if q["gamma_u"] <= gu and q["gamma_p"] <= gp]
            q = min(ok, key=lambda q: q["wu"]) if ok else None
            best.append({"bounds": [gu, gp], "n_meeting": len(ok), **(q or {"s": None})})
            q1 = min([q for q in ok if q["s"][3] == 1], key=lambda q: q["wu"], default=None)
            best_k1.append({"bounds": [gu, gp], **(q1 or {"s": None})})
            qt = min(ok, key=lambda q: q["ms"]) if ok else None
            fastest.append({"bounds": [gu, gp], **(qt or {"s": None})})
        out[f"P2P1_L{L}"] = {"dofs": info.n_dofs, "omega_inv": om, "err_disc": e_disc, "tuples": len(rows),
                             "minimal_wu": best, "minimal_wu_kappa1": best_k1, "fastest": fastest,
                             "under_10_wu": [q["s"] is not None and q["wu"] < 10 for q in best]}
        if args.rows_out:
            with open(f"{args.rows_out}_L{L}.json", "w") as f:
                json.dump(rows, f)
        del pb, x
        torch.cuda.empty_cache()
    dt = time.perf_counter() - t0
    print(json.dumps({"metric": "minimal W(FMG(s)) at disc.-error accuracy (Sec. 5.1 search space S)",
                      "value": dt, "unit": "s (whole study)", "n_gpus": 1, "higher_is_better": False,
                      "dtype": "f32+f64", "data": "synthetic",
                      "config": {"workload": "P2-P1, 6-tet cube, paper's cube solution, coarse level 2, levels 6 "
                                             "and 7, FP32 V-cycles in FP64 refinement, 768 tuples per level",
                                 "results": out}}))


def run_reference(args):
    """The reference arm: the CPU oracle as it stands on every host core, one
    independent FMG of the level-4 sample of the workload per core per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prm = dict(PARAMS, omega_inv=0.32)
    cores, model = _host_cpu()
    times, dofs = [], 0
    with _oracle_pool(cores, prm, CPU_SAMPLE_LEVEL) as pool:
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            res = pool.map(_oracle_fmg, range(cores))
            if i >= args.warmup:
                times.append(time.perf_counter() - t0)
            dofs = res[0][1]
    t = statistics.median(times)
    v = cores * dofs / t
    w = WORKLOAD
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "DoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{w['disc']} Stokes, 6-macro-tet cube, oracle sample at level {CPU_SAMPLE_LEVEL} "
                                   f"of the level-{w['L']} workload, one solve per host core per step",
                       "params": PARAMS},
            "cpu_baseline": {"value": v, "unit": "DoF/s", "cores": cores, "kind": "oracle",
                             "sample": f"level {CPU_SAMPLE_LEVEL} ({dofs} DoF) FMG on each of {cores} single-threaded "
                                       f"processes per step, host {model}"},
            "e2e": {"value": v, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def learned_coarse(pb, wl, prm, steps, warmup, stream):
    """Learned coarse-grid correction against the plain coarse solve on the
    same FMG: training pairs are coarse defects recorded from V-cycles of
    random-forcing problems (seeded) plus random defects; targets from the
    plain dense coarse solve; training on the GPU by the library's own
    forward/backward kernels.  Then the gated FMG (network accepted only if
    its coarse residual passes the gate) and the network alone."""
    import torch
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    L, lc = WORKLOAD["L"], WORKLOAD["lc"]
    lr = min(lc + 2, L)
    pb.nn_record(True)
    for seed in range(100):
        hhg.set_workload_rhs(pb, Workload("modes", seed=7000 + seed), levels=range(lc, lr + 1))
        xx = pb.new_vector(lr)
        for _ in range(5):
            pb.vcycle(lr, prm, xx, pb.level_vector(lr, "rhs"))
    recorded = pb.nn_record(False)
    hhg.set_workload_rhs(pb, wl)
    rep = pb.nn_train(epochs=60, batch=256, lr=1e-3, n_train=9500, seed=2, recorded=True, smooth_frac=0.5)
    out = {"n": rep.n, "params": rep.n_params, "recorded_defects": recorded, "loss_first": rep.loss_first,
           "loss_last": rep.loss_last, "val_rel_err": rep.val_rel_err, "train_ms": rep.train_ms, "theta": 0.1}
    x = pb.new_vector(L)
    for mode, name in ((1, "gated"), (2, "network_only")):
        pb.nn_enable(mode, theta=0.1)
        pb.fmg_solve(prm, x, stats=False)
        pb.nn_counts()
        tt = statistics.mean(time_steps(pb, prm, x, steps, warmup, stream)) * 1e-3
        acc, rej = pb.nn_counts()
        # gamma of this FMG's solution x against the discrete solution, which
        # the plain coarse solve computes
        pb.nn_enable(0)
        if bool(torch.isfinite(x).all()):
            gg = accuracy(pb, wl, prm, x)
        else:
            gg = (None, None)           # the FMG diverged
        out[name] = {"ms_per_step": tt * 1e3, "gamma_u": gg[0], "gamma_p": gg[1], "accepted": acc, "rejected": rej}
    return out


def bound_report(gu, gp):
    """Which (gamma_u, gamma_p) bound pairs the solve meets."""
    return {"disc_bound": list(DISC_BOUND), "disc_accuracy": bool(gu <= DISC_BOUND[0] and gp <= DISC_BOUND[1]),
            "table3_bounds_met": [list(bd) for bd in TABLE3_BOUNDS if gu <= bd[0] and gp <= bd[1]]}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="hhg", choices=["hhg", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--workload", default="p2-l7", choices=["p2-l7", "p2-l6", "batched", "p1-visc", "tme", "tme-disc"])
    ap.add_argument("--rows-out", default="", help="tme-disc: write every tuple's row to <prefix>_L<level>.json")
    ap.add_argument("--profile-region", action="store_true",
                    help="only set-up, warm-up and the timed FMG steps, bracketed by cudaProfilerStart/Stop")
    ap.add_argument("--profile-e2e", action="store_true",
                    help="only set-up and one end-to-end step (host data in, FMG, solution out), bracketed by "
                         "cudaProfilerStart/Stop")
    ap.add_argument("--profile-apply", action="store_true",
                    help="only the FP32 apply of the roofline line (or, with --workload p1-visc, the level-7 "
                         "P1-P1 apply), bracketed by cudaProfilerStart/Stop")
    args = ap.parse_args()
    if args.workload in WORKLOADS:
        WORKLOAD.clear()
        WORKLOAD.update(WORKLOADS[args.workload])
    if args.profile_apply:
        return profile_apply(args.workload)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "p1-visc":
        return run_p1_visc(args)
    if args.workload == "tme":
        return run_tme(args)
    if args.workload == "tme-disc":
        return run_tme_disc(args)

    import torch
    import torch.distributed as dist
    from paper_2010_13513_gb300 import hhg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    # a created stream: the library records whole FMG solves as CUDA graphs on it
    torch.cuda.set_stream(torch.cuda.Stream())
    if world > 1:
        dist.init_process_group("nccl")
    hhg.load()
    L = WORKLOAD["L"]
    learned = rank == 0 and not args.no_learned and not args.profile_region and not args.profile_e2e

    # ---------------- set-up (not timed): hierarchy, rhs on all levels, omega
    pb, wl = make_problem("mixed", error_level=(rank == 0 and not args.profile_region and not args.profile_e2e), nn=learned)
    shapes = pb.autotune(reps=5)
    if args.profile_e2e:
        e2e_steps(pb, wl, hhg.Params.make(**PARAMS, omega_inv=0.32), 1, profile=True)
        return
    if args.profile_region:
        prm = hhg.Params.make(**PARAMS, omega_inv=0.32)
        x = pb.new_vector(L)
        for _ in range(args.warmup):
            pb.fmg_solve(prm, x, stats=False)
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        for _ in range(args.steps):
            pb.fmg_solve(prm, x, stats=False)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        return
    om = omega_inv(pb)
    prm = hhg.Params.make(**PARAMS, omega_inv=om)
    stream = pb.stream
    x = pb.new_vector(L)
    st = pb.fmg_solve(prm, x)
    launches = st.kernel_launches
    acc = accuracy(pb, wl, prm, x) if rank == 0 else None

    # ---------------- timed region
    sampler = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    times = time_steps(pb, prm, x, args.steps, args.warmup, stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    t_step = statistics.mean(times) * 1e-3
    if world > 1:
        tt = torch.tensor([t_step], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_step = float(tt.item())
    dofs = pb.layout(L).n_dofs
    value = world * dofs / t_step
    if rank != 0:
        dist.destroy_process_group()
        return

    # the same mixed solve with the FP64 refinement residual instead of the
    # double-float one (the default): its time and the solutions' difference
    refine = {"kind": pb.refinement_residual_kind()}
    if refine["kind"] == "df32":
        xf = pb.new_vector(L)
        pb.set_refinement_residual("fp64")
        tf = statistics.mean(time_steps(pb, prm, xf, max(3, args.steps // 2), 2, stream)) * 1e-3
        pb.set_refinement_residual("df32")
        refine.update({"fp64_refinement_ms_per_step": tf * 1e3, "df32_speedup": tf / t_step,
                       "rel_diff_vs_fp64_refinement": float(torch.linalg.norm(x - xf) / torch.linalg.norm(xf))})
        del xf

    # FP64-only GPU solve of the same workload (same tuple, same omega)
    pb64, _ = make_problem("fp64")
    pb64.autotune(reps=3)
    x64 = pb64.new_vector(L)
    t64 = statistics.mean(time_steps(pb64, prm, x64, max(3, args.steps // 2), 2, pb64.stream)) * 1e-3
    mixed_vs_fp64 = float(torch.linalg.norm(x - x64) / torch.linalg.norm(x64))
    del pb64, x64

    alg_bytes, t_apply = apply_roofline(pb)
    pk, src = peaks()
    achieved = alg_bytes / t_apply / 1e9
    # wall-clock steps on a shared host: an occasional step stalls for tens of
    # ms outside the library (seen as isolated 56-94 ms steps among 28.5 ms
    # ones), so the value is the median step; the mean and every step are
    # reported beside it
    e2e_t, h2d, d2h = e2e_steps(pb, wl, prm, max(3, min(args.steps, 7)))
    e2e_v = dofs / statistics.median(e2e_t)
    nn = learned_coarse(pb, wl, prm, max(3, args.steps // 2), 2, stream) if learned else None
    sh = pb.launch_shape(L)
    traffic = measured_traffic(sh)
    line = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"P2-P1 Taylor-Hood Stokes, 6-macro-tet unit cube, level {L}, analytic cube solution "
                               f"of Sec. 5.1.1, coarse level {WORKLOAD['lc']}, FMG with FP32 V-cycles in FP64 "
                               "iterative refinement",
                   "dofs": dofs, "params": PARAMS, "omega_inv": om, "coarse_level": WORKLOAD["lc"],
                   "l2": "flushed (512 MB write) before every timed step; level-7 vectors exceed L2",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "gamma_u": acc[0], "gamma_p": acc[1], **bound_report(acc[0], acc[1]),
                   "err_fmg": acc[2], "err_disc": acc[3], "disc_solve_cycles": acc[4],
                   "wu_model": st.wu_model, "wu_counted": st.wu_counted, "wu_target": 10.0,
                   "wu_model_under_target": bool(st.wu_model < 10.0),
                   "launch_shapes": {str(k): v for k, v in shapes.items()},
                   "fp64_gpu_ms_per_step": t64 * 1e3, "mixed_speedup_vs_fp64_gpu": t64 / t_step,
                   "mixed_vs_fp64_rel_diff": mixed_vs_fp64, "refinement_residual": refine,
                   "learned_coarse": nn},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / pk["hbm_gbs"], "traffic": traffic,
                     "traffic_source": (f"carried over from the committed ncu summary "
                                        f"{TRAFFIC_PROFILE.format(disc=WORKLOAD['disc'].lower(), L=L)} "
                                        f"(DRAM bytes of one apply; taken on the same kernel sources, "
                                        f"sha256 {kernel_source_hash()[:12]}..., and the same apply shape "
                                        f"{[sh[3], sh[4]]})") if traffic is not None else None,
                     "kernel": f"FP32 operator apply y = calA x, level {L} (FULL; launch shape {list(sh)})",
                     "alg_bytes": alg_bytes, "avg_launch_us": t_apply * 1e6, "peak_source": src},
        "e2e": {"value": e2e_v, "unit": "DoF/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "statistic": "median step", "mean_value": dofs / statistics.mean(e2e_t),
                "step_ms": [t * 1e3 for t in e2e_t]},
        "gpu_launches": launches * args.steps,
        "clocks": clocks,
    }
    if not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(dict(PARAMS, omega_inv=om))
    print(json.dumps(line))


if __name__ == "__main__":
    main()
