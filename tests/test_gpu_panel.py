"""The paper's own operator on the GPU (cubed-sphere panel, Eq. (14), native FP64) against the panel
oracle: the library's geometry against the oracle's (two implementations from the definition), every
kernel on several levels and shapes (ragged against the 32 x 4 thread tiles, nz odd and 1), and
multigrid solves -- same cycles as the oracle, iterates within 1e-10 -- on a small panel and on the
paper's 512^2 x 128 configuration (5 levels, V(1,1), rho = 2/3, epsilon = 1e-5), and the fused
line-preconditioned CG against the oracle's PCG."""
import numpy as np
import pytest
import torch

import oracle
from oracle import panel as opanel
from paper_1402_3545_gb300 import tpmg, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-10  # relative 2-norm, the FP64 application tolerance

SHAPES = [(96, 72, 33, 3), (64, 40, 16, 2), (40, 24, 1, 2), (128, 128, 8, 4)]


def rel(a, b):
    a, b = np.ravel(a), np.ravel(b)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def _pair(nx, ny, nz, L, om2=None, lam2=1.0, H=0.01):
    om2 = (4.2 * 0.5 * np.pi / nx) ** 2 if om2 is None else om2
    op = tpmg.PanelOperator(nx, ny, nz, om2, lam2, H, nlevels=L)
    ref = opanel.PanelProblem(nx, ny, nz, L, om2, lam2, H)
    return op, ref


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_geometry_matches_the_oracle(shape):
    nx, ny, nz, L = shape
    op, ref = _pair(nx, ny, nz, L)
    for l in range(1, L + 1):
        nzl, nyl, nxl = op.level_shape(l)
        got = tpmg.panel_level_geometry(op.op, l, nxl, nyl)
        for g, r in zip(got, ref.geo(l)):
            assert g.shape == r.shape and rel(g, r) < 1e-13
    op.close()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
def test_kernels_match_the_oracle_on_every_level(shape):
    nx, ny, nz, L = shape
    op, ref = _pair(nx, ny, nz, L)
    rng = np.random.default_rng(nx + ny + nz)
    for l in range(1, L + 1):
        sh = op.level_shape(l)
        n = int(np.prod(sh))
        u, f = rng.standard_normal(sh), rng.standard_normal(sh)
        ud, fd = dev(u), dev(f)
        out = torch.empty_like(ud)
        tpmg.panel_apply_A(op.op, l, ud, out, n)
        assert rel(host(out), ref.apply_A(u, l)) < TOL
        tpmg.panel_line_solve(op.op, l, fd, out, n)
        assert rel(host(out), ref.line_solve(f, l)) < TOL
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.panel_residual(op.op, l, ud, fd, out, n, norm_out=nrm)
        r_ref = ref.residual(u, f, l)
        assert rel(host(out), r_ref) < TOL
        assert abs(nrm.item() - np.linalg.norm(r_ref)) < TOL * np.linalg.norm(r_ref)
        tpmg.panel_smooth(op.op, l, 0.8, ud, fd, out, n, norm_out=nrm)
        assert rel(host(out), u + 0.8 * ref.line_solve(r_ref, l)) < TOL
        assert abs(nrm.item() - np.linalg.norm(r_ref)) < TOL * np.linalg.norm(r_ref)
        if l < L:  # RestrictSmooth onto level l from level l + 1, Prolongate from level l into l + 1
            shf = op.level_shape(l + 1)
            nf = int(np.prod(shf))
            rf = rng.standard_normal(shf)
            fc, uc = torch.empty_like(ud), torch.empty_like(ud)
            tpmg.panel_restrict_smooth(op.op, l, 0.7, dev(rf), fc, uc, nf, n)
            fc_ref = opanel.restrict(rf)
            assert rel(host(fc), fc_ref) < TOL
            assert rel(host(uc), 0.7 * ref.line_solve(fc_ref, l)) < TOL
            uf = rng.standard_normal(shf)
            ufd = dev(uf)
            tpmg.panel_prolongate(op.op, l + 1, ud, ufd, n, nf)
            assert rel(host(ufd), opanel.prolongate_add(u, uf)) < TOL
    op.close()


@pytest.mark.parametrize("nu", [(1, 1), (2, 2)], ids=["V11", "V22"])
def test_multigrid_matches_the_oracle(nu):
    nx, ny, nz, L = 64, 64, 32, 4
    op, ref = _pair(nx, ny, nz, L)
    f = np.random.default_rng(11).standard_normal((nz, ny, nx))
    u_ref, it_ref, hist_ref, conv = ref.mg_solve(f, tol=1e-8, max_iter=60, nu_pre=nu[0], nu_post=nu[1],
                                                 rho=2.0 / 3.0)
    assert conv
    u = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    prm = tpmg.default_params(prec=tpmg.F64, tol=1e-8, max_iter=60, nu_pre=nu[0], nu_post=nu[1], rho=2.0 / 3.0,
                              zero_guess=1)
    res = tpmg.mg_solve(op.op, prm, dev(f).reshape(-1), u, f.size)
    assert res["iters"] == it_ref
    # the residual of an iterate that differs from the oracle's by rounding (~1e-16) moves by up to
    # kappa(A) ~ 4e5 times that relative to ||f||: compare the history while it is well above that
    h, hr = np.asarray(res["history"]), np.asarray(hist_ref)
    big = hr > 1e-5
    assert np.allclose(h[big], hr[big], rtol=1e-6, atol=0)
    assert rel(host(u), u_ref) < TOL
    op.close()


def test_cg_matches_the_oracle():
    """Line-preconditioned CG with the fused panel kernels: the oracle's textbook PCG is the same
    iteration (the lagged update is algebraically equal), so the counts agree within one and the first
    twenty relative residuals to 1e-6."""
    nx, ny, nz = 64, 48, 32
    op, ref = _pair(nx, ny, nz, 1)
    f = np.random.default_rng(12).standard_normal((nz, ny, nx))
    u_ref, it_ref, hist_ref, conv = ref.cg_solve(f, tol=1e-8, max_iter=500)
    assert conv
    u = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    res = tpmg.cg_solve(op.op, tpmg.default_params(prec=tpmg.F64, tol=1e-8, max_iter=500, zero_guess=1),
                        dev(f).reshape(-1), u, f.size)
    assert res["converged"] and abs(res["iters"] - it_ref) <= 1
    assert np.allclose(res["history"][:20], hist_ref[:20], rtol=1e-6)
    if res["iters"] == it_ref:  # the same number of steps of the same iteration: rounding apart only
        assert rel(host(u), u_ref) < 1e-6
    r = ref.residual(host(u).reshape(f.shape), f)
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-8 * 1.01
    op.close()


def test_panel_refuses_other_precisions():
    op, _ = _pair(32, 32, 4, 2)
    f = torch.zeros(32 * 32 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="native FP64"):
        tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.DW), f, torch.zeros_like(f), f.numel())
    op.close()


@pytest.mark.parametrize("tol", [1e-6, 1e-10])
def test_mixed_precision_solve(tol):
    """Iterative refinement on the panel: FP64 outer residual, FP32 V-cycles. The residual of its
    solution, recomputed by the oracle, meets the tolerance; at 1e-10 the solution is within 1e-6 of
    the oracle's multigrid solve to 1e-12 (the final-solution bound); the cycle count stays within two
    of the FP64 multigrid's (the inner cycle is the same iteration in FP32)."""
    nx, ny, nz, L = 128, 96, 32, 4
    op, ref = _pair(nx, ny, nz, L)
    f = np.random.default_rng(13).standard_normal((nz, ny, nx))
    fd = dev(f).reshape(-1)
    u = torch.zeros(f.size, dtype=torch.float64, device="cuda")
    prm = dict(tol=tol, max_iter=80, nu_pre=1, nu_post=1, rho=2.0 / 3.0, zero_guess=1)
    res = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.MIXED, **prm), fd, u, f.size)
    assert res["converged"], res
    uh = host(u).reshape(f.shape)
    assert np.linalg.norm(ref.residual(uh, f)) / np.linalg.norm(f) < tol * 1.01
    u64 = torch.zeros_like(u)
    r64 = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.F64, **prm), fd, u64, f.size)
    assert abs(res["iters"] - r64["iters"]) <= 2, (res["iters"], r64["iters"])
    if tol <= 1e-10:
        before = oracle.set_threads(0)
        oracle.set_threads(64)
        try:
            u_star, _, _, _ = ref.mg_solve(f, tol=1e-12, max_iter=200, nu_pre=1, nu_post=1, rho=2.0 / 3.0)
        finally:
            oracle.set_threads(before)
        assert rel(uh, u_star) < 1e-6
    op.close()


def test_flat_entry_points_refuse_a_panel_operator():
    """The flat-box entry points need the flat operator's buffers: given a panel operator they return
    TPMG_ERR_ARG instead of touching memory the panel operator does not have."""
    op, _ = _pair(64, 64, 4, 2)
    n = op.level_n(2)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    for call in (lambda: tpmg.apply_A(op.op, 2, tpmg.F64, x, x.clone(), n),
                 lambda: tpmg.smooth(op.op, 2, tpmg.F64, 0.8, x, x, x.clone(), n),
                 lambda: tpmg.autotune(op.op, tpmg.F64, op.L),
                 lambda: tpmg.time_kernel(op.op, tpmg.F64, tpmg.K_SMOOTH)):
        with pytest.raises(tpmg.TpmgError) as e:
            call()
        assert e.value.status == tpmg.ERR_ARG
    op.close()


def test_paper_configuration_full_size():
    """512^2 x 128 on a whole cube face, the paper's solver settings: the GPU's cycles and iterate
    equal the oracle's (all host threads), and the residual recomputed by the oracle meets epsilon."""
    p = workloads.panel()
    f = p.rhs()
    before = oracle.set_threads(0)
    oracle.set_threads(64)
    try:
        ref = opanel.PanelProblem(p.nx, p.ny, p.nz, p.nlevels, p.omega2, p.lambda2, p.H, p.extent)
        u_ref, it_ref, _, conv = ref.mg_solve(f, tol=1e-5, max_iter=60, nu_pre=1, nu_post=1, rho=2.0 / 3.0)
        assert conv
        op = tpmg.PanelOperator(p.nx, p.ny, p.nz, p.omega2, p.lambda2, p.H, p.extent, nlevels=p.nlevels)
        u = torch.zeros(p.n, dtype=torch.float64, device="cuda")
        prm = tpmg.default_params(prec=tpmg.F64, tol=1e-5, max_iter=60, nu_pre=1, nu_post=1, rho=2.0 / 3.0,
                                  zero_guess=1)
        res = tpmg.mg_solve(op.op, prm, dev(f).reshape(-1), u, p.n)
        assert res["iters"] == it_ref
        uh = host(u).reshape(f.shape)
        assert rel(uh, u_ref) < TOL
        r = ref.residual(uh, f)
        assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-5
        op.close()
    finally:
        oracle.set_threads(before)
