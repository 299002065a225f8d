"""Full-size checks in the bench's launch configuration (512 x 512 x 128, varying lambda^2, 7 levels):
the FP64-accurate solve takes the oracle's iteration count and residual history
(tests/golden/oracle_counts.txt, written by a script that calls only the oracle), and every final
solution's residual is recomputed on the host by the oracle's operator. Plus a mid-size mixed solve
run twice: bit-identical results (no races, fixed-order reductions)."""
import os

import numpy as np
import pytest
import torch

import oracle
from helpers import read_golden
from paper_1402_3545_gb300 import autotune, tpmg, workloads

pytestmark = pytest.mark.gpu


def _golden_history(name):
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_counts.txt")
    for line in open(path):
        if line.startswith(f"# {name}:") and "history" in line:
            vals = line.split("history", 1)[1].split("(")[0].split()
            return np.array([float(x) for x in vals])
    raise KeyError(name)


@pytest.fixture(scope="module")
def mid():
    p = workloads.mid()
    f = p.rhs()
    op = tpmg.Operator.from_problem(p)
    autotune.tune(op, tpmg.DW, lambda_varies=True)
    yield p, f, op
    op.close()


def test_dw_solve_full_size_matches_oracle_history(mid):
    p, f, op = mid
    g = read_golden("oracle_counts.txt")
    fd = torch.from_numpy(f).cuda()
    u = torch.zeros_like(fd)
    res = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.DW, tol=1e-6), fd, u, p.n)
    assert res["converged"] and res["iters"] == int(g["mid_iters"])
    assert np.allclose(res["history"], _golden_history("mid"), rtol=2e-3)  # golden printed to 4 digits
    cx, cy, v = oracle.problem_coefficients(p)
    r = oracle.residual(u.cpu().numpy(), f, cx, cy, v)
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-6


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_mixed_solve_full_size(mid, tol):
    p, f, op = mid
    fd = torch.from_numpy(f).cuda()
    u = torch.zeros_like(fd)
    res = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.MIXED, tol=tol, max_iter=60), fd, u, p.n)
    assert res["converged"], res
    cx, cy, v = oracle.problem_coefficients(p)
    r = oracle.residual(u.cpu().numpy(), f, cx, cy, v)
    assert np.linalg.norm(r) / np.linalg.norm(f) < tol * 1.001


def test_mixed_solve_is_deterministic_mid_size():
    p = workloads.scaled_down(workloads.mid(), 256, 256, 128)
    f = torch.from_numpy(p.rhs()).cuda()
    op = tpmg.Operator.from_problem(p)
    runs = []
    for _ in range(2):
        u = torch.zeros_like(f)
        res = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.MIXED, tol=1e-8, max_iter=60), f, u, p.n)
        assert res["converged"], res
        runs.append((u.cpu().numpy(), res["history"]))
    assert np.array_equal(runs[0][0], runs[1][0]) and runs[0][1] == runs[1][1]
    op.close()
