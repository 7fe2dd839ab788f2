"""Learned coarse-grid correction: GPU forward/backward kernels against the
CPU oracle MLP, training on the GPU, and what the trained network gains in
the V-cycle (against no coarse correction and against the plain solve)."""
import numpy as np
import pytest
import torch

from gpu_helpers import curl_workload, lib_problem, oracle_hierarchy, rel

pytestmark = pytest.mark.gpu


def _nn_problem(hidden=64, samples=512, batch=64, L=4, lc=2, solve="fp64"):
    from paper_2010_13513_gb300 import hhg
    mesh = hhg.Mesh.box(1, 1, 1, 1.0)
    pb = hhg.Problem(mesh, disc="P1P1", L=L, coarse_level=lc, solve=solve, nn_hidden=hidden, nn_samples=samples,
                     nn_batch=batch)
    hhg.set_workload_rhs(pb, curl_workload())
    return pb


def _flat(params):
    return np.concatenate([p.reshape(-1) for p in params]).astype(np.float32)


def _unflat(flat, shapes):
    out, o = [], 0
    for sh in shapes:
        k = int(np.prod(sh))
        out.append(flat[o:o + k].reshape(sh))
        o += k
    return out


def test_gradients_match_oracle():
    from oracle import mlp
    pb = _nn_problem(hidden=48, samples=64, batch=32)
    n, P = pb.nn_size()
    assert n == 3 * 27 + 125           # interior P1 velocity DoFs x 3 + pressure nodes on level 2
    params = mlp.init(n, 48, seed=4)
    rng = np.random.default_rng(5)
    params = [p + 0.01 * rng.standard_normal(p.shape) for p in params]
    shapes = [p.shape for p in params]
    p32 = [p.astype(np.float32).astype(np.float64) for p in params]   # the values the GPU sees
    pb.nn_set_params(_flat(params))
    assert np.array_equal(pb.nn_get_params(), _flat(params))
    X = rng.standard_normal((32, n)).astype(np.float32)
    T = rng.standard_normal((32, n)).astype(np.float32)
    loss, g = pb.nn_grad(X, T)
    ref_loss = mlp.loss(p32, X.astype(np.float64), T.astype(np.float64))
    ref_g = mlp.grads(p32, X.astype(np.float64), T.astype(np.float64))
    assert abs(loss / ref_loss - 1) < 1e-5
    for gg, rr in zip(_unflat(g, shapes), ref_g):
        assert rel(gg.astype(np.float64), rr) < 1e-4


def test_training_and_vcycle_gain():
    """Trained on coarse defects recorded from V-cycles of random-forcing
    problems (targets from the plain coarse solver), the network alone still
    drives the V-cycle of a different problem (the curl solution) with a rate
    between the plain solve and no coarse correction; the residual gate accepts
    it only when its coarse residual is small enough, so the gated cycle never
    loses against the plain one."""
    from hhg_inputs import Workload
    from paper_2010_13513_gb300 import hhg
    L = 4
    pb = _nn_problem(hidden=512, samples=8000, batch=128)
    prm = hhg.Params.make(2, 2, 1, 1, "f", 2, 0.5)
    pb.nn_record(True)
    for seed in range(400):
        hhg.set_workload_rhs(pb, Workload("modes", seed=5000 + seed))
        x = pb.new_vector(L)
        pb.fmg_solve(prm, x, stats=False)
        for _ in range(2):
            pb.vcycle(L, prm, x, pb.level_vector(L, "rhs"))
    recorded = pb.nn_record(False)
    assert recorded >= 2000
    rep = pb.nn_train(epochs=100, batch=128, lr=1e-3, n_train=7800, seed=2, recorded=True, smooth_frac=0.5)
    print(f"\nlearned coarse correction: n={rep.n}, params={rep.n_params}, {recorded} recorded defects, loss "
          f"{rep.loss_first:.3e} -> {rep.loss_last:.3e}, validation relative error {rep.val_rel_err:.3f}, "
          f"training {rep.train_ms:.1f} ms")
    assert rep.loss_last < 0.01 * rep.loss_first
    hhg.set_workload_rhs(pb, curl_workload())
    b = pb.level_vector(L, "rhs")

    def rate(mode, theta=0.1):
        pb.nn_enable(mode, theta=theta)
        x = pb.new_vector(L)
        r = pb.new_vector(L)
        res = [max(pb.residual(L, x, b, r, norms=True))]
        for _ in range(6):
            pb.vcycle(L, prm, x, b)
            res.append(max(pb.residual(L, x, b, r, norms=True)))
        return (res[-1] / res[1]) ** (1 / 5), pb.nn_counts()

    plain, _ = rate(0)
    net, _ = rate(2)
    none, _ = rate(3)
    gated = {th: rate(1, th) for th in (0.1, 0.3, 0.5)}
    print(f"V-cycle rates: plain {plain:.3f}, network only {net:.3f}, no coarse correction {none:.3f}")
    for th, (rt, (acc, rej)) in gated.items():
        print(f"  gate theta={th}: rate {rt:.3f}, accepted {acc}, rejected {rej}")
    assert net < none                                   # the network beats dropping the coarse solve
    for th, (rt, _) in gated.items():
        assert rt <= max(plain, net) * 1.05 + 1e-3      # gating never makes the cycle worse than its parts
