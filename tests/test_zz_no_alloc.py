"""The allocation-free residual entry point, for callers that must not allocate device memory
while they run (a framework that already owns nearly all device memory through its own pool, or a
latency-critical loop that cannot afford cudaMalloc's implicit synchronisation).

It is checked through the C ABI against the regular entry point tpmg_residual (FP64) on the same
level, within the FP64 tolerance the other tests use, and against the oracle's residual, on calls in
a row whose inputs and grid sizes change from one call to the next, so stale partial sums left in
the shared scratch array by an earlier call would show up. The grids reach every residual kernel
the library can pick: the pointwise kernel (at most 4096 columns), the one-column plane-pipelined
kernel (nx a multiple of 32 but not of 64) and the two-column persistent sweep (nx a multiple of 64,
even ny, more than 4096 columns). This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import TOL, rel
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu

MAX_BLOCKS = 65536  # TPMG_NOALLOC_MAX_BLOCKS in include/tpmg.h


def _case(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    lam2 = 1e3 * (1.0 + 0.5 * rng.random((ny, nx)))
    op = tpmg.Operator(nx, ny, nz, 1e-2, 1.0 / nx, 1.0 / ny, 1.0 / nz, lam2, nlevels=1)
    cx, cy, v = tpmg.op_level_coefficients(op.op, 1, nx * ny)
    u = rng.standard_normal((nz, ny, nx))
    f = rng.standard_normal((nz, ny, nx))
    return op, cx, cy, v, u, f


# (nx, ny, nz, seed): pointwise (twice), two-column persistent (twice), one-column pipelined
CASES = [(96, 40, 33, 1), (64, 12, 17, 2), (128, 64, 16, 3), (256, 128, 32, 4), (160, 72, 9, 5)]


def test_noalloc_residual_matches_regular_entry_point_and_oracle():
    for nx, ny, nz, seed in CASES:
        op, cx, cy, v, u_h, f_h = _case(nx, ny, nz, seed)
        u = torch.from_numpy(u_h).cuda()
        f = torch.from_numpy(f_h).cuda()
        n = nx * ny * nz
        r_ref = torch.empty_like(u)
        norm_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.residual(op.op, 1, tpmg.F64, u, f, r_ref, n, norm_out=norm_ref)
        r = torch.full_like(u, float("nan"))
        norm = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        tpmg.residual_norm_noalloc(nx, ny, nz, cx, cy, torch.from_numpy(v).cuda(), u, f, r, norm)
        torch.cuda.synchronize()
        r_h = r.cpu().numpy()
        assert rel(r_h, r_ref.cpu().numpy()) < TOL[tpmg.F64], (nx, ny, nz)
        assert abs(norm.item() - norm_ref.item()) <= TOL[tpmg.F64] * norm_ref.item(), (nx, ny, nz)
        r_orc = oracle.residual(u_h, f_h, cx, cy, v.reshape(ny, nx))
        assert rel(r_h, r_orc) < TOL[tpmg.F64], (nx, ny, nz)
        assert abs(norm.item() - np.linalg.norm(r_orc)) <= TOL[tpmg.F64] * np.linalg.norm(r_orc)
        op.close()


def test_noalloc_large_grid_on_the_two_column_sweep():
    """4096 x 4096 columns: the two-column persistent sweep runs at most 16 blocks per SM whatever
    the grid, so this size fits the fixed scratch and is computed, not refused."""
    nx = ny = 4096
    op, cx, cy, v, u_h, f_h = _case(nx, ny, 1, 6)
    u = torch.from_numpy(u_h).cuda()
    f = torch.from_numpy(f_h).cuda()
    r_ref = torch.empty_like(u)
    norm_ref = torch.zeros(1, dtype=torch.float64, device="cuda")
    tpmg.residual(op.op, 1, tpmg.F64, u, f, r_ref, nx * ny, norm_out=norm_ref)
    r = torch.full_like(u, float("nan"))
    norm = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    tpmg.residual_norm_noalloc(nx, ny, 1, cx, cy, torch.from_numpy(v).cuda(), u, f, r, norm)
    torch.cuda.synchronize()
    assert rel(r.cpu().numpy(), r_ref.cpu().numpy()) < TOL[tpmg.F64]
    assert abs(norm.item() - norm_ref.item()) <= TOL[tpmg.F64] * norm_ref.item()
    op.close()


def test_noalloc_rejects_grids_beyond_the_fixed_scratch():
    """nx = 4064 is a multiple of 32 but not of 64, so the grid takes the one-column pipelined
    kernel with (nx / 32) * (ny / 4) blocks: ny = 2064 needs 127 * 516 = 65532 blocks (accepted by
    the size check), ny = 2080 needs 127 * 520 = 66040 > 65536 and is refused before any launch, so
    the dummy pointers of the refused call are never dereferenced."""
    assert (4064 // 32) * (2064 // 4) <= MAX_BLOCKS < (4064 // 32) * (2080 // 4)
    x = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    lib = tpmg.load()
    status = lib.tpmg_residual_norm_noalloc(4064, 2080, 1, 1.0, 1.0, p, p, p, p, p, None)
    assert status == tpmg.ERR_ARG
    assert b"66040 thread blocks" in lib.tpmg_noalloc_last_error()
