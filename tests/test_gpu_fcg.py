"""Flexible CG on the GPU against the oracle's FCG(1): with the V-cycle preconditioner alone, with
a network that never helps (every learned correction rejected, iteration unchanged bit for bit),
and with an affine network whose corrections are accepted, for one- and two-channel inputs.

The GPU preconditioner is an FP32 V-cycle and the oracle's an FP64 one. Each application differs
by the FP32 line solves' relative error, at most t = 4 u_32 kappa(M) (gpu_common.tol_inverse; about
9e-5 on this problem's stiff columns), and the differences add up along the recurrence, so
history entry k is held to 4 k t; iteration counts agree to +-1; the final iterate is checked with
the oracle's FP64 residual."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import dev, host, make_problem, tol_inverse
from helpers import affine_network
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module")
def prob():
    p = make_problem(64, 64, 32)
    op = tpmg.Operator.from_problem(p)
    cx, cy, v = oracle.problem_coefficients(p)
    f = p.rhs()
    yield p, op, (cx, cy, v), f
    op.close()


def run_gpu(op, p, f, nn=None, aux=None, tol=TOL, max_iter=200):
    prm = tpmg.default_params(tol=tol, max_iter=max_iter)
    u = torch.zeros(p.nz, p.ny, p.nx, dtype=torch.float64, device="cuda")
    res = tpmg.fcg_solve(op.op, prm, dev(f, tpmg.F64), u, p.n, nn=nn, aux=aux)
    return host(u), res


def check_solution(u, f, cx, cy, v, tol=TOL):
    r = oracle.residual(u, f, cx, cy, v)
    assert np.linalg.norm(r) / np.linalg.norm(f) < tol * 1.01


def test_fcg_vcycle_matches_oracle(prob):
    p, op, (cx, cy, v), f = prob
    u, res = run_gpu(op, p, f)
    _, it, hist, conv, _, _ = oracle.fcg_solve(f, cx, cy, v, mode=1, nlevels=op.L, tol=TOL, max_iter=200)
    assert conv and res["converged"]
    assert abs(res["iters"] - it) <= 1, (res["iters"], it)
    t = tol_inverse(tpmg.F32, cx, cy, v)
    for k in range(1, min(5, it, res["iters"]) + 1):
        assert abs(res["history"][k] / hist[k] - 1.0) < 4 * k * t, (k, res["history"][k], hist[k], t)
    check_solution(u, f, cx, cy, v)


def test_zero_network_is_always_rejected(prob):
    """A zero network returns zero, the learned correction equals z1 and is never kept: the
    iteration is the V-cycle-only one, bit for bit."""
    p, op, (cx, cy, v), f = prob
    _, base = run_gpu(op, p, f)
    net = tpmg.Network(1)
    u, res = run_gpu(op, p, f, nn=net)
    assert res["nn_accepted"] == 0
    assert res["iters"] == base["iters"] and res["history"] == base["history"]
    check_solution(u, f, cx, cy, v)
    net.close()


@pytest.mark.parametrize("bad", ["nan", "huge"])
def test_corrupted_network_falls_back(prob, bad):
    """Corrupted weights (NaN, or 1e30 so that the output overflows) give non-finite or useless
    corrections; every one is rejected and the iteration is the V-cycle-only one, bit for bit."""
    p, op, (cx, cy, v), f = prob
    _, base = run_gpu(op, p, f)
    params = np.full(tpmg.nn_nparams(1), np.nan if bad == "nan" else 1e30, dtype=np.float32)
    net = tpmg.Network(1, params)
    u, res = run_gpu(op, p, f, nn=net)
    assert res["nn_accepted"] == 0
    assert res["iters"] == base["iters"] and res["history"] == base["history"]
    check_solution(u, f, cx, cy, v)
    net.close()


@pytest.fixture(scope="module")
def prob_small():
    p = make_problem(64, 32, 16)
    op = tpmg.Operator.from_problem(p)
    cx, cy, v = oracle.problem_coefficients(p)
    f = p.rhs()
    yield p, op, (cx, cy, v), f
    op.close()


@pytest.mark.parametrize("cin", [1, 2])
def test_affine_network_matches_oracle(prob_small, cin):
    """With NN(x) = alpha x0 + beta (+ gamma relu(x1)) the learned correction D^-1 NN is a damped
    Jacobi step (alpha = 1/8) plus a small constant; both sides accept it and converge in the same
    number of iterations (+-1)."""
    p, op, (cx, cy, v), f = prob_small
    params = affine_network(cin, 0.125, 1e-3, gamma=2.0 ** -14 if cin == 2 else 0.0)
    aux = np.random.default_rng(5).uniform(0.0, 1.0, (p.ny, p.nx))
    net = tpmg.Network(cin, params.astype(np.float32))
    u, res = run_gpu(op, p, f, nn=net,
                     aux=torch.from_numpy(aux.astype(np.float32).ravel()).cuda() if cin == 2 else None)
    ref_aux = aux.astype(np.float32).astype(np.float64) if cin == 2 else None
    _, it, hist, conv, used, rejected = oracle.fcg_solve(f, cx, cy, v, mode=2, nlevels=op.L, tol=TOL,
                                                         max_iter=200, params=params, aux=ref_aux)
    assert conv and res["converged"]
    assert used > 0
    assert abs(res["iters"] - it) <= 1, (res["iters"], it)
    assert abs(res["nn_accepted"] - used) <= 1, (res["nn_accepted"], used)
    k = min(3, it, res["iters"]) + 1
    assert np.allclose(res["history"][:k], hist[:k], rtol=1e-2, atol=0)
    check_solution(u, f, cx, cy, v)
    net.close()


def test_fcg_argument_errors(prob):
    p, op, _, f = prob
    net = tpmg.Network(2)
    with pytest.raises(tpmg.TpmgError):
        run_gpu(op, p, f, nn=net)  # a 2-channel network without its aux field
    net.close()
    q = make_problem(96, 32, 8)
    op2 = tpmg.Operator.from_problem(q)
    net1 = tpmg.Network(1)
    with pytest.raises(tpmg.TpmgError):
        run_gpu(op2, q, q.rhs(), nn=net1)  # nx not a multiple of 64
    # without a network any grid is fine
    u, res = run_gpu(op2, q, q.rhs())
    assert res["converged"]
    net1.close()
    op2.close()


def test_fcg_zero_rhs_and_max_iter(prob):
    p, op, _, f = prob
    u, res = run_gpu(op, p, np.zeros_like(f))
    assert res["converged"] and res["iters"] == 0 and not np.any(u)
    _, res = run_gpu(op, p, f, tol=1e-14, max_iter=2)
    assert res["status"] == tpmg.ERR_NOT_CONVERGED and res["iters"] == 2


def test_fcg_zero_guess_ignores_u(prob):
    """zero_guess = 1 on a u full of NaN gives bit for bit the solve from u = 0."""
    p, op, _, f = prob
    u0, r0 = run_gpu(op, p, f)
    prm = tpmg.default_params(tol=TOL, max_iter=200, zero_guess=1)
    u = torch.full((p.nz, p.ny, p.nx), float("nan"), dtype=torch.float64, device="cuda")
    r1 = tpmg.fcg_solve(op.op, prm, dev(f, tpmg.F64), u, p.n)
    assert r1["iters"] == r0["iters"] and r1["history"] == r0["history"]
    assert np.array_equal(host(u), u0)
