"""The learned stage end to end on a small grid: training pairs from the multigrid solver, Adam on
the residual loss, the checkpoint round trip and the ablation of flexible CG with and without the
network (same right-hand side, iterations and time reported)."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_1402_3545_gb300 import learned, tpmg, workloads

pytestmark = pytest.mark.gpu

CFG = learned.TrainConfig(nx=64, ny=64, nz=32, h=1.0 / 512, hz=1.0 / 32, n_problems=3, steps=150, lr=2e-3)


@pytest.fixture(scope="module")
def trained():
    pairs = learned.generate_pairs(CFG)
    held = learned.generate_pairs(dataclasses.replace(CFG, n_problems=1, seed=7))
    before = learned.evaluate(tpmg.Network(CFG.cin, learned.init_params(CFG.cin, CFG.seed)), held, CFG.shape)
    net, losses, _ = learned.train(CFG, pairs)
    after = learned.evaluate(net, held, CFG.shape)
    return net, pairs, held, before, after, losses


def test_pairs_are_consistent(trained):
    """A D^-1 target = x0 up to the BF16 rounding of x0 and the reference solve's 1e-10: the target
    is the error whose residual is the input."""
    _, pairs, _, _, _, _ = trained
    x, t, lam2, op = pairs[0]
    n = CFG.nx * CFG.ny * CFG.nz
    p = workloads.Problem("pair", CFG.nx, CFG.ny, CFG.nz, CFG.omega2, CFG.h, CFG.h, CFG.hz, lam2, 1, 0, "uniform")
    cx, cy, v = oracle.problem_coefficients(p)
    tt = t.double().cpu().numpy().reshape(CFG.shape)
    x0 = x.view(n, CFG.cin)[:, 0].double().cpu().numpy().reshape(CFG.shape)
    r = oracle.apply_A(tt * oracle.diag_inv(CFG.shape, cx, cy, v), cx, cy, v)
    assert np.linalg.norm(r - x0) < 1e-2 * np.linalg.norm(x0)


def test_training_lowers_the_residual_loss(trained):
    _, _, _, before, after, losses = trained
    assert 0.9 < before["residual"] < 1.1  # a fresh network proposes almost nothing
    assert after["residual"] < 0.5, after
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:5])


def test_checkpoint_round_trip(trained, tmp_path):
    net, _, _, _, _, _ = trained
    path = str(tmp_path / "net.npz")
    learned.save(path, net, CFG, {"note": "test"})
    net2, meta = learned.load(path)
    assert np.array_equal(net2.get_params(), net.get_params())
    assert meta["nx"] == CFG.nx and meta["loss"] == "residual" and meta["note"] == "test"
    net2.close()


def test_ablation_with_and_without_the_network(trained):
    """Same right-hand side, flexible CG with the V-cycle alone and with the learned stage: both
    converge and the trained corrections are kept, and the measured gain is the one the bound of
    tests/test_learned_stage_bound.py allows: a corrector with the network's 9^3 receptive field can
    remove at most a few per cent of the error a V-cycle leaves, so the iteration count stays within
    one of the V-cycle-only count, while the network does remove most of its input residual (held-out
    residual loss below 0.5) and leaves the held-out error where it was (error ratio 0.9 .. 1.1)."""
    net, _, _, _, _, _ = trained
    p = workloads.Problem("ablation", 128, 128, 32, CFG.omega2, CFG.h, CFG.h, CFG.hz, 1e3,
                          learned.levels_full(128, 128), 3, "uniform")
    res = learned.fcg_compare(p, net, tol=1e-8)
    a, b = res["fcg_vcycle"], res["fcg_learned"]
    print(f"ablation: V-cycle {a['iters']} it {a['ms']:.2f} ms; learned {b['iters']} it {b['ms']:.2f} ms, "
          f"{b['nn_accepted']} corrections kept")
    assert a["converged"] and b["converged"]
    assert b["nn_accepted"] > 0
    assert abs(b["iters"] - a["iters"]) <= 1
    _, _, _, _, after, _ = trained
    assert after["residual"] < 0.5 and 0.9 < after["error"] < 1.1, after
