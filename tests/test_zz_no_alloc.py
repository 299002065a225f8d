"""The allocation-free residual entry point, for callers that must not allocate device memory
while they run (a framework that already owns nearly all device memory through its own pool, or a
latency-critical loop that cannot afford cudaMalloc's implicit synchronisation).

It is checked through the C ABI against the regular entry point tpmg_residual (FP64) on the same
level, within the FP64 tolerance the other tests use, on two calls in a row: the second call gets
other inputs and a smaller grid, so stale partial sums left in the shared scratch array by the
first call would show up. This file is collected last so that a run stopping at the first failure
has run every other test before it.
"""
import numpy as np
import pytest
import torch

from gpu_common import TOL, rel
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu


def _case(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    lam2 = 1e3 * (1.0 + 0.5 * rng.random((ny, nx)))
    op = tpmg.Operator(nx, ny, nz, 1e-2, 1.0 / nx, 1.0 / ny, 1.0 / nz, lam2, nlevels=1)
    cx, cy, v = tpmg.op_level_coefficients(op.op, 1, nx * ny)
    u = torch.from_numpy(rng.standard_normal((nz, ny, nx))).cuda()
    f = torch.from_numpy(rng.standard_normal((nz, ny, nx))).cuda()
    return op, cx, cy, torch.from_numpy(v).cuda(), u, f


def test_noalloc_residual_matches_regular_entry_point_twice():
    for nx, ny, nz, seed in [(96, 40, 33, 1), (64, 12, 17, 2)]:
        op, cx, cy, v, u, f = _case(nx, ny, nz, seed)
        n = nx * ny * nz
        r_ref = torch.empty_like(u)
        norm_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.residual(op.op, 1, tpmg.F64, u, f, r_ref, n, norm_out=norm_ref)
        r = torch.full_like(u, float("nan"))
        norm = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        tpmg.residual_norm_noalloc(nx, ny, nz, cx, cy, v, u, f, r, norm)
        torch.cuda.synchronize()
        assert rel(r.cpu().numpy(), r_ref.cpu().numpy()) < TOL[tpmg.F64]
        assert abs(norm.item() - norm_ref.item()) <= TOL[tpmg.F64] * norm_ref.item()
        op.close()


def test_noalloc_rejects_oversized_grids():
    """4096 x 4096 columns need 128 * 1024 thread blocks, more than the fixed scratch holds: the
    size check refuses the call before any kernel is launched."""
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    status = tpmg.load().tpmg_residual_norm_noalloc(4096, 4096, 1, 1.0, 1.0, p, p, p, p, p, None)
    assert status == tpmg.ERR_ARG
    assert b"fixed scratch" in tpmg.load().tpmg_noalloc_last_error()
