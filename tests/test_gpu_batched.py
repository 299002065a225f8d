"""The batched persistent solver: problems of different sizes and levels solved in one cooperative
launch, checked problem by problem against the oracle; convergence masks; the grid barrier's time
limit (a zero limit makes the waits run out: the solve reports TPMG_ERR_TIMEOUT and the device stays
usable)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1402_3545_gb300 import tpmg, workloads

pytestmark = pytest.mark.gpu


def small_batch(n=7, seed=3):
    """Problems shaped like the batched workload (sizes drawn per problem, lambda^2 log-uniform in
    [1e2, 1e4], uniform RHS) but small enough for the oracle: nx, ny in {32, 64}, nz in {8, 16, 32}."""
    rng = np.random.default_rng(seed)
    probs = []
    for b in range(n):
        nx = int(rng.choice([32, 64]))
        ny = int(rng.choice([32, 64]))
        nz = int(rng.choice([8, 16, 32]))
        lam2 = float(10 ** rng.uniform(2, 4))
        h = 1.0 / max(nx, ny)  # square horizontal cells, as in the batched workload
        probs.append(workloads.Problem(f"b{b}", nx, ny, nz, 1e-2, h, h, 1.0 / nz, lam2,
                                       workloads.levels_to_8(nx, ny), 1000 + b, "uniform"))
    return probs


def run_batch(probs, fs=None, **kw):
    ops = [tpmg.Operator.from_problem(p) for p in probs]
    fs = [torch.from_numpy(p.rhs()).cuda() for p in probs] if fs is None else fs
    us = [torch.zeros_like(f) for f in fs]
    prm = tpmg.default_params(prec=tpmg.MIXED, **kw)
    res = tpmg.mg_solve_batched([o.op for o in ops], prm, fs, us)
    return ops, fs, us, res


def test_batched_matches_oracle_problem_by_problem():
    probs = small_batch()
    ops, fs, us, res = run_batch(probs, tol=1e-8, max_iter=60)
    assert res["status"] == tpmg.OK
    for p, f, u, r in zip(probs, fs, us, res["problems"]):
        cx, cy, v = oracle.problem_coefficients(p)
        fh = f.cpu().numpy()
        assert r["converged"]
        rr = oracle.residual(u.cpu().numpy(), fh, cx, cy, v)
        assert np.linalg.norm(rr) / np.linalg.norm(fh) < 1e-8 * 1.001
        # the same iteration as the oracle's multigrid (linear cycle): counts agree within one
        _, it_ref, _, _ = oracle.mg_solve(fh, cx, cy, v, p.nlevels, tol=1e-8, max_iter=60)
        assert abs(r["iters"] - it_ref) <= 1, (p.name, r["iters"], it_ref)
    for o in ops:
        o.close()


def test_batched_equals_single_problem_solves():
    """Each problem of the batch reaches what the single-problem mixed solver reaches."""
    probs = small_batch(4, seed=9)
    ops, fs, us, res = run_batch(probs, tol=1e-6)
    for p, o, f, u, r in zip(probs, ops, fs, us, res["problems"]):
        u1 = torch.zeros_like(f)
        single = tpmg.mg_solve(o.op, tpmg.default_params(prec=tpmg.MIXED, tol=1e-6), f, u1, p.n)
        assert abs(single["iters"] - r["iters"]) <= 1
        err = (u - u1).norm().item() / u1.norm().item()
        assert err < 1e-5
    for o in ops:
        o.close()


def test_batched_masks_converged_and_zero_problems():
    probs = small_batch(3, seed=11)
    fs = [torch.from_numpy(p.rhs()).cuda() for p in probs]
    fs[1].zero_()  # converged before the first cycle
    ops, fs, us, res = run_batch(probs, fs=fs, tol=1e-6)
    pr = res["problems"]
    assert pr[1]["converged"] and pr[1]["iters"] == 0 and not us[1].any()
    assert pr[0]["converged"] and pr[2]["converged"]
    # max_iter reached: reported, iterate kept
    for o in ops:
        o.close()
    ops, fs, us, res = run_batch(probs, tol=1e-14, max_iter=2)
    assert res["status"] == tpmg.ERR_NOT_CONVERGED
    assert all(r["iters"] == 2 and not r["converged"] for r in res["problems"])
    for o in ops:
        o.close()


def test_barrier_time_limit_reports_timeout_and_device_stays_usable():
    probs = small_batch(3, seed=13)
    ops = [tpmg.Operator.from_problem(p) for p in probs]
    fs = [torch.from_numpy(p.rhs()).cuda() for p in probs]
    us = [torch.zeros_like(f) for f in fs]
    prm = tpmg.default_params(prec=tpmg.MIXED, timeout_s=0.0)
    with pytest.raises(tpmg.TpmgError) as e:
        tpmg.mg_solve_batched([o.op for o in ops], prm, fs, us)
    assert e.value.status == tpmg.ERR_TIMEOUT
    # the context is intact: the same batch with the default limit converges
    for u in us:
        u.zero_()
    res = tpmg.mg_solve_batched([o.op for o in ops], tpmg.default_params(prec=tpmg.MIXED), fs, us)
    assert res["status"] == tpmg.OK and all(r["converged"] for r in res["problems"])
    for o in ops:
        o.close()


def test_batched_argument_errors():
    probs = small_batch(2, seed=17)
    ops = [tpmg.Operator.from_problem(p) for p in probs]
    fs = [torch.from_numpy(p.rhs()).cuda() for p in probs]
    us = [torch.zeros_like(f) for f in fs]
    with pytest.raises(tpmg.TpmgError) as e:
        tpmg.mg_solve_batched([o.op for o in ops], tpmg.default_params(prec=tpmg.DW), fs, us)
    assert e.value.status == tpmg.ERR_ARG
    with pytest.raises(tpmg.TpmgError):
        tpmg.mg_solve_batched([ops[0].op, ops[0].op], tpmg.default_params(prec=tpmg.MIXED), [fs[0], fs[0]],
                              [us[0], us[0]])
    for o in ops:
        o.close()


def test_batched_zero_guess_ignores_u():
    """zero_guess = 1 on fields full of NaN gives bit for bit the batched solve from u = 0 (the same
    operators, so the kept tables are reused and only the captured graph changes)."""
    probs = small_batch(3, seed=13)
    ops, fs, us, res = run_batch(probs, tol=1e-6)
    us2 = [torch.full_like(f, float("nan")) for f in fs]
    res2 = tpmg.mg_solve_batched([o.op for o in ops], tpmg.default_params(prec=tpmg.MIXED, tol=1e-6, zero_guess=1),
                                 fs, us2)
    for a, b, u, u2 in zip(res["problems"], res2["problems"], us, us2):
        assert a["iters"] == b["iters"] and a["history"] == b["history"]
        assert torch.equal(u, u2)
    for o in ops:
        o.close()


def test_batched_fused_residual_restrict_equals_separate_tasks():
    """The batched cycle's fused Residual + RestrictSmooth tasks (levels 64 columns wide and more)
    give bit for bit the solve with separate Residual and RestrictSmooth tasks."""
    rng = np.random.default_rng(21)
    probs = []
    for b, (nx, ny, nz) in enumerate([(64, 64, 16), (128, 64, 32), (64, 32, 8), (32, 64, 16)]):
        lam2 = float(10 ** rng.uniform(2, 4))
        h = 1.0 / max(nx, ny)
        probs.append(workloads.Problem(f"f{b}", nx, ny, nz, 1e-2, h, h, 1.0 / nz, lam2,
                                       workloads.levels_to_8(nx, ny), 2000 + b, "uniform"))
    ops, fs, us, res = run_batch(probs, tol=1e-8, max_iter=60)
    for o in ops:
        tpmg.set_fusion(o.op, False)
    us2 = [torch.zeros_like(f) for f in fs]
    res2 = tpmg.mg_solve_batched([o.op for o in ops], tpmg.default_params(prec=tpmg.MIXED, tol=1e-8, max_iter=60),
                                 fs, us2)
    for a, b, u, u2 in zip(res["problems"], res2["problems"], us, us2):
        assert a["converged"] and a["iters"] == b["iters"] and a["history"] == b["history"]
        assert torch.equal(u, u2)
    for o in ops:
        o.close()
