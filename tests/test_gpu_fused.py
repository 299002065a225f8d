"""GPU parity of the fused Residual + RestrictSmooth pass (Algorithm 1: the kernels "Residual" and
"RestrictSmooth" of Sec. 3.1 in one sweep over the fine level, the fine residual never stored)
against the FP64 oracle, its equality with the two separate kernels, and the multigrid solver with
and without the fusion (same iterations, residual history and iterate, bit for bit).

The fused kernel applies where the fine level has nx % 64 == 0 and even ny and the coarse level
more than 4096 columns (smaller ones solve their columns by cyclic reduction); the shapes below
give one such level pair each (192 x 96 -> 96 x 48 with three 64-column tiles per row, 256 x 128
-> 128 x 64) and one pair below it that takes the separate kernels. nz = 1 and 7 sit below the
kernel's four-plane ring; a constant lambda^2 exercises the per-plane factor tables.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import PREC_IDS, PRECS, TOL, dev, host, make_problem, oracle_levels, rel, tol_inverse
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu

SHAPES = [(192, 96, 20, None), (256, 128, 7, None), (256, 128, 1, None), (192, 96, 33, 1e3)]
SHAPE_IDS = [f"{a}x{b}x{c}" + ("" if d is None else "_const") for a, b, c, d in SHAPES]

@pytest.fixture(scope="module", params=SHAPES, ids=SHAPE_IDS)
def setup(request):
    nx, ny, nz, lam = request.param
    p = make_problem(nx, ny, nz, lam=lam)
    op = tpmg.Operator.from_problem(p)  # coarsened down to 8 columns across, as the solver runs
    cx, cy, v = oracle.problem_coefficients(p)
    lv = oracle_levels(cx, cy, v, op.L)
    yield op, lv, p
    tpmg.set_fusion(op.op, True)
    op.close()


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def fused_applies(op, level) -> bool:
    nz, nyf, nxf = op.level_shape(level + 1)
    _, nyc, nxc = op.level_shape(level)
    return nxf % 64 == 0 and nyf % 2 == 0 and nxc * nyc > 4096


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_residual_restrict_smooth_vs_oracle(setup, prec):
    """f_c = R (f - A u) and u_c = rho M_c^{-1} f_c against the oracle's residual, restriction and
    line solve, on every level pair."""
    op, lv, p = setup
    rho = 0.8
    for level in range(1, op.L):
        u, f = rnd(op.level_shape(level + 1), 100 + level), rnd(op.level_shape(level + 1), 110 + level)
        td = dev(u, prec).dtype
        fc = torch.empty(op.level_shape(level), dtype=td, device="cuda")
        uc = torch.empty_like(fc)
        tpmg.residual_restrict_smooth(op.op, level, prec, rho, dev(u, prec), dev(f, prec), fc, uc,
                                      op.level_n(level + 1), op.level_n(level))
        f_ref = oracle.restrict(oracle.residual(u, f, *lv[level + 1]))
        u_ref = rho * oracle.line_solve(f_ref, *lv[level])
        assert rel(host(fc), f_ref) < TOL[prec], (level, rel(host(fc), f_ref))
        assert rel(host(uc), u_ref) < tol_inverse(prec, *lv[level]), (level, rel(host(uc), u_ref))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_fused_equals_separate_kernels(setup, prec):
    """One launch where the fused kernel applies; the same values as tpmg_residual followed by
    tpmg_restrict_smooth (bit for bit in FP64 and FP32; in double-word the separate calls round the
    residual to FP64 in between)."""
    op, lv, p = setup
    rho = 0.8
    for level in range(1, op.L):
        u = dev(rnd(op.level_shape(level + 1), 120 + level), prec)
        f = dev(rnd(op.level_shape(level + 1), 130 + level), prec)
        nf, nc = op.level_n(level + 1), op.level_n(level)
        fc = torch.empty(op.level_shape(level), dtype=u.dtype, device="cuda")
        uc = torch.empty_like(fc)
        torch.cuda.synchronize()
        k0 = tpmg.kernel_launches()
        tpmg.residual_restrict_smooth(op.op, level, prec, rho, u, f, fc, uc, nf, nc)
        launches = tpmg.kernel_launches() - k0
        if prec != tpmg.DW:
            assert launches == (1 if fused_applies(op, level) else 2), (level, launches)
        r = torch.empty_like(u)
        fc2, uc2 = torch.empty_like(fc), torch.empty_like(fc)
        tpmg.residual(op.op, level + 1, prec, u, f, r, nf)
        tpmg.restrict_smooth(op.op, level, prec, rho, r, fc2, uc2, nf, nc)
        torch.cuda.synchronize()
        if prec == tpmg.DW:
            assert rel(host(fc), host(fc2)) < 1e-13 and rel(host(uc), host(uc2)) < 1e-13
        else:
            assert torch.equal(fc, fc2) and torch.equal(uc, uc2), level


@pytest.mark.parametrize("prec", [tpmg.F64, tpmg.DW, tpmg.F32, tpmg.MIXED], ids=["f64", "dw", "f32", "mixed"])
def test_mg_solve_same_with_and_without_fusion(setup, prec):
    """The solver's V-cycles with the fused pass reproduce those with the two kernels exactly."""
    op, lv, p = setup
    f = rnd(op.level_shape(op.L), 7)
    fd = dev(f, tpmg.F32 if prec == tpmg.F32 else tpmg.F64)
    tol = 1e-4 if prec == tpmg.F32 else 1e-8
    out = {}
    for fuse in (True, False):
        tpmg.set_fusion(op.op, fuse)
        u = torch.zeros_like(fd)
        res = tpmg.mg_solve(op.op, tpmg.default_params(prec=prec, tol=tol, max_iter=40), fd, u, p.n)
        torch.cuda.synchronize()
        out[fuse] = (res, u)
    tpmg.set_fusion(op.op, True)
    a, ua = out[True]
    b, ub = out[False]
    assert a["iters"] == b["iters"] and a["history"] == b["history"], (a["iters"], b["iters"])
    assert torch.equal(ua, ub)
    # the iterate meets the tolerance, its residual recomputed with the oracle's operator (nz = 1 has
    # no vertical coupling: point smoothing of a horizontally anisotropic problem, too slow for 40
    # cycles)
    if p.nz > 1:
        cx, cy, v = lv[op.L]
        r = np.linalg.norm(oracle.residual(host(ua), f, cx, cy, v)) / np.linalg.norm(f)
        assert a["converged"] and r < 2 * tol, (a["iters"], r)
