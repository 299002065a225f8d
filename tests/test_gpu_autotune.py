"""Tile variants of the pipelined Smooth and the autotuner: every variant gives the same per-cell
result, the tuner returns valid choices and the JSON cache replays them."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, make_problem
from paper_1402_3545_gb300 import autotune, tpmg

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(128, 64, 32), (32, 160, 5), (256, 130, 64)], ids=["128x64x32", "32x160x5", "256x130x64"])
@pytest.mark.parametrize("prec", [tpmg.DW, tpmg.F32, tpmg.F64], ids=["dw", "f32", "f64"])
def test_variants_give_identical_smoothing(prec, shape):
    """Every tile variant (shared-memory stack, persistent with global scratch) gives the
    same smoothed field bit for bit; the shapes include a one-tile-wide level (periodic wrap onto the
    same tile), a short column and a y extent that is not a multiple of 4."""
    nx, ny, nz = shape
    p = make_problem(nx, ny, nz)
    op = tpmg.Operator.from_problem(p, nlevels=2)
    rng = np.random.default_rng(5)
    u, f = dev(rng.standard_normal((nz, ny, nx)), prec), dev(rng.standard_normal((nz, ny, nx)), prec)
    outs, norms = [], []
    for v in range(tpmg.NUM_VARIANTS):
        tpmg.set_variant(op.op, prec, 2, v)
        o = torch.empty_like(u)
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.smooth(op.op, 2, prec, 0.8, u, f, o, p.n, norm_out=nrm)
        outs.append(host(o))
        norms.append(host(nrm)[0])
    for o, nv in zip(outs[1:], norms[1:]):
        assert np.array_equal(o, outs[0])
        assert abs(nv - norms[0]) <= 1e-6 * norms[0]
    op.close()


def test_autotune_and_cache(tmp_path, monkeypatch):
    monkeypatch.setenv("TPMG_TUNE_CACHE", str(tmp_path / "tuning.json"))
    p = make_problem(128, 128, 64)
    op = tpmg.Operator.from_problem(p)
    first = autotune.tune(op, tpmg.DW, lambda_varies=True, reps=2)
    assert len(first) == op.L and all(0 <= v < tpmg.NUM_VARIANTS for v in first)
    again = autotune.tune(op, tpmg.DW, lambda_varies=True)
    assert again == first
    # the tuned operator still solves exactly like the oracle-checked default schedule
    f = dev(p.rhs(), tpmg.DW)
    u = torch.zeros_like(f)
    res = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.DW), f, u, p.n)
    assert res["converged"]
    op.close()
