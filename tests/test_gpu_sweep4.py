"""The FP32 Smooth and line solve with one 128 x ROWS tile per warp (four columns x ROWS rows per thread,
Thomas factors 1/m_k formed in registers): the same per-cell arithmetic as the two-column sweep, so
the smoothed field equals variant 5's bit for bit -- on one-tile and many-wave grids, nz from 1 to
128, lambda^2 varying by column (per-cell factors, converged range) or constant (shared table) --
and the line solve meets the FP32 forward-error bound against the oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import dev, host, make_problem, rel, tol_inverse
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu

SHAPES = [(128, 2, 1), (128, 4, 2), (256, 6, 3), (384, 10, 17), (128, 64, 33), (512, 32, 128), (2048, 200, 4)]
X4_VARIANTS = range(8, tpmg.NUM_VARIANTS)


@pytest.mark.parametrize("lam", [None, 1e3], ids=["varying", "constant"])
@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_four_column_smooth_equals_two_column(shape, lam):
    nx, ny, nz = shape
    p = make_problem(nx, ny, nz, lam=lam)
    op = tpmg.Operator.from_problem(p, nlevels=2)
    rng = np.random.default_rng(nx + ny + nz)
    u = dev(rng.standard_normal((nz, ny, nx)), tpmg.F32)
    f = dev(rng.standard_normal((nz, ny, nx)), tpmg.F32)

    def run(variant):
        tpmg.set_variant(op.op, tpmg.F32, 2, variant)
        o = torch.empty_like(u)
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.smooth(op.op, 2, tpmg.F32, 0.8, u, f, o, p.n, norm_out=nrm)
        return host(o), host(nrm)[0]

    ref, nref = run(5)
    for v in X4_VARIANTS:
        o, nv = run(v)
        assert np.array_equal(o, ref), (v, np.max(np.abs(o - ref)))
        assert abs(nv - nref) <= 1e-6 * nref
    op.close()


@pytest.mark.parametrize("lam", [None, 1e3], ids=["varying", "constant"])
@pytest.mark.parametrize("shape", [(128, 2, 1), (256, 6, 3), (384, 10, 17), (128, 64, 33)],
                         ids=lambda s: "x".join(map(str, s)))
def test_four_column_line_solve_matches_oracle(shape, lam):
    nx, ny, nz = shape
    p = make_problem(nx, ny, nz, lam=lam)
    op = tpmg.Operator.from_problem(p, nlevels=2)
    cx, cy, v = oracle.problem_coefficients(p)
    b = np.random.default_rng(7).standard_normal((nz, ny, nx))
    x = torch.empty(p.n, dtype=torch.float32, device="cuda")
    tpmg.line_solve(op.op, 2, tpmg.F32, dev(b, tpmg.F32), x, p.n)
    ref = oracle.line_solve(b.astype(np.float32).astype(np.float64), cx, cy, v)
    assert rel(host(x).reshape(b.shape), ref) < tol_inverse(tpmg.F32, cx, cy, v)
    op.close()
