"""GPU parity of every kernel of the hot path against the FP64 oracle, element by element, on
seeded inputs that span several 32-wide warps, several blocks and ragged tails in x and y.

Called through the C ABI (libtpmg.so) via the thin binding; compared with oracle/ (plain C).
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import PREC_IDS, PRECS, TOL, dev, host, make_problem, oracle_levels, rel, tol_inverse
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu

# (nx, ny, nz, nlevels): ragged x (not a multiple of 32), ragged y, odd nz, single column height
# levels of at most 4096 columns run the cell-parallel kernels (parallel cyclic reduction), larger
# ones the column kernels (pipelined when nx % 32 == 0): 100 x 50 exercises the plain column
# kernels on its finest level; nz = 7, 9, 200 are not powers of two; nz = 256 is the largest
# kernels, and 128 x 48 (6144 columns, nx % 64 == 0) the plane-pipelined Smooth, the two-column
# Residual and the 2 x 2 prolongation on its finest level
SHAPES = [(80, 36, 24, 3), (64, 64, 64, 4), (40, 12, 7, 3), (96, 8, 1, 2), (16, 16, 128, 2), (100, 50, 9, 2),
          (16, 4, 200, 2), (8, 8, 256, 2), (128, 48, 20, 2)]
SHAPE_IDS = [f"{a}x{b}x{c}L{d}" for a, b, c, d in SHAPES]


@pytest.fixture(scope="module", params=SHAPES, ids=SHAPE_IDS)
def setup(request):
    nx, ny, nz, L = request.param
    p = make_problem(nx, ny, nz)
    op = tpmg.Operator.from_problem(p, nlevels=L)
    cx, cy, v = oracle.problem_coefficients(p)
    lv = oracle_levels(cx, cy, v, L)
    yield op, lv, p
    op.close()


def rnd(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_apply_A(setup, prec):
    op, lv, p = setup
    for level in range(1, op.L + 1):
        sh = op.level_shape(level)
        x = rnd(sh, 1 + level)
        y = torch.empty_like(dev(x, prec))
        tpmg.apply_A(op.op, level, prec, dev(x, prec), y, op.level_n(level))
        ref = oracle.apply_A(x, *lv[level])
        assert rel(host(y), ref) < TOL[prec], (level, rel(host(y), ref))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_line_solve(setup, prec):
    op, lv, p = setup
    for level in range(1, op.L + 1):
        sh = op.level_shape(level)
        b = rnd(sh, 10 + level)
        x = torch.empty_like(dev(b, prec))
        tpmg.line_solve(op.op, level, prec, dev(b, prec), x, op.level_n(level))
        ref = oracle.line_solve(b, *lv[level])
        assert rel(host(x), ref) < tol_inverse(prec, *lv[level]), (level, rel(host(x), ref))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_smooth_with_fused_norm(setup, prec):
    op, lv, p = setup
    rho = 0.8
    for level in range(1, op.L + 1):
        sh = op.level_shape(level)
        u, f = rnd(sh, 20 + level), rnd(sh, 30 + level)
        out = torch.empty_like(dev(u, prec))
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.smooth(op.op, level, prec, rho, dev(u, prec), dev(f, prec), out, op.level_n(level), norm_out=nrm)
        ref = oracle.smooth(u, f, *lv[level], rho)
        assert rel(host(out), ref) < tol_inverse(prec, *lv[level]), (level, rel(host(out), ref))
        rnorm = np.linalg.norm(oracle.residual(u, f, *lv[level]))
        assert abs(host(nrm)[0] - rnorm) / rnorm < max(TOL[prec], 1e-7)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_residual_with_fused_norm(setup, prec):
    op, lv, p = setup
    for level in range(1, op.L + 1):
        sh = op.level_shape(level)
        u, f = rnd(sh, 40 + level), rnd(sh, 50 + level)
        r = torch.empty_like(dev(u, prec))
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.residual(op.op, level, prec, dev(u, prec), dev(f, prec), r, op.level_n(level), norm_out=nrm)
        ref = oracle.residual(u, f, *lv[level])
        assert rel(host(r), ref) < TOL[prec], (level, rel(host(r), ref))
        assert abs(host(nrm)[0] - np.linalg.norm(ref)) / np.linalg.norm(ref) < max(TOL[prec], 1e-7)


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_restrict_smooth(setup, prec):
    op, lv, p = setup
    rho = 0.8
    for level in range(1, op.L):
        rf = rnd(op.level_shape(level + 1), 60 + level)
        fc = torch.empty(op.level_shape(level), dtype=dev(rf, prec).dtype, device="cuda")
        uc = torch.empty_like(fc)
        tpmg.restrict_smooth(op.op, level, prec, rho, dev(rf, prec), fc, uc, op.level_n(level + 1), op.level_n(level))
        f_ref = oracle.restrict(rf)
        u_ref = rho * oracle.line_solve(f_ref, *lv[level])
        assert rel(host(fc), f_ref) < TOL[prec]
        assert rel(host(uc), u_ref) < tol_inverse(prec, *lv[level]), (level, rel(host(uc), u_ref))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_prolongate(setup, prec):
    op, lv, p = setup
    for level in range(2, op.L + 1):
        uc = rnd(op.level_shape(level - 1), 70 + level)
        uf = rnd(op.level_shape(level), 80 + level)
        t = dev(uf, prec)
        tpmg.prolongate(op.op, level, prec, dev(uc, prec), t, op.level_n(level - 1), op.level_n(level))
        ref = oracle.prolongate_add(uc, uf)
        assert rel(host(t), ref) < TOL[prec], (level, rel(host(t), ref))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
def test_cg_fused_kernels(setup, prec):
    """Fused SpMV and fused Tridiag (Sec. 3.1) against their definitions applied with the oracle's
    operator and line solve."""
    op, lv, p = setup
    L = op.L
    sh = op.level_shape(L)
    n = op.level_n(L)
    u, pp, z, q, r = (rnd(sh, 90 + s) for s in range(5))
    alpha, beta = 0.37, 0.61
    tu, tp, tz, tq = dev(u, prec), dev(pp, prec), dev(z, prec), dev(q, prec)
    sigma = torch.zeros(1, dtype=torch.float64, device="cuda")
    tpmg.cg_fused_spmv(op.op, prec, alpha, beta, tu, tp, tz, tq, sigma, n)
    u_ref = u + alpha * pp
    p_ref = z + beta * pp
    q_ref = oracle.apply_A(z, *lv[L]) + beta * q
    assert rel(host(tu), u_ref) < TOL[prec]
    assert rel(host(tp), p_ref) < TOL[prec]
    assert rel(host(tq), q_ref) < TOL[prec]
    s_ref = float(np.sum(p_ref * q_ref))
    assert abs(host(sigma)[0] - s_ref) <= max(TOL[prec], 1e-7) * np.linalg.norm(p_ref) * np.linalg.norm(q_ref)

    tr, tq2, tz2 = dev(r, prec), dev(q, prec), torch.empty_like(dev(r, prec))
    rr = torch.zeros(1, dtype=torch.float64, device="cuda")
    rz = torch.zeros(1, dtype=torch.float64, device="cuda")
    tpmg.cg_fused_tridiag(op.op, prec, alpha, tr, tq2, tz2, rr, rz, n)
    r_ref = r - alpha * q
    z_ref = oracle.line_solve(r_ref, *lv[L])
    assert rel(host(tr), r_ref) < TOL[prec]
    assert rel(host(tz2), z_ref) < tol_inverse(prec, *lv[L])
    assert abs(host(rr)[0] - np.sum(r_ref ** 2)) / np.sum(r_ref ** 2) < max(TOL[prec], 1e-7)
    rz_ref = float(np.sum(r_ref * z_ref))
    assert abs(host(rz)[0] - rz_ref) <= max(tol_inverse(prec, *lv[L]), 1e-7) * np.linalg.norm(r_ref) * np.linalg.norm(z_ref)


def test_deterministic_reductions(setup):
    """Two identical applications give bit-identical outputs and norms (fixed-order reductions)."""
    op, lv, p = setup
    L = op.L
    sh = op.level_shape(L)
    u, f = dev(rnd(sh, 5), tpmg.DW), dev(rnd(sh, 6), tpmg.DW)
    outs, norms = [], []
    for _ in range(2):
        o = torch.empty_like(u)
        nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
        tpmg.smooth(op.op, L, tpmg.DW, 0.8, u, f, o, op.level_n(L), norm_out=nrm)
        outs.append(host(o))
        norms.append(host(nrm)[0])
    assert np.array_equal(outs[0], outs[1]) and norms[0] == norms[1]


def test_argument_errors(setup):
    op, lv, p = setup
    sh = op.level_shape(op.L)
    x = dev(rnd(sh, 7), tpmg.F64)
    y = torch.empty_like(x)
    with pytest.raises(tpmg.TpmgError) as e:
        tpmg.apply_A(op.op, op.L + 1, tpmg.F64, x, y, op.level_n(op.L))
    assert e.value.status == tpmg.ERR_ARG
    with pytest.raises(tpmg.TpmgError):
        tpmg.prolongate(op.op, 1, tpmg.F64, x, y, op.level_n(op.L), op.level_n(op.L))
    with pytest.raises(TypeError):
        tpmg.apply_A(op.op, op.L, tpmg.F32, x, y, op.level_n(op.L))


@pytest.mark.parametrize("prec", PRECS, ids=PREC_IDS)
@pytest.mark.parametrize("variant", range(tpmg.NUM_VARIANTS))
def test_every_smooth_variant_matches_oracle(prec, variant):
    """Each tile variant of the large-level Smooth (shared-memory stack, persistent with the stack
    in global scratch, two columns per thread) against the oracle, with its fused norm."""
    nx, ny, nz = 128, 48, 20
    p = make_problem(nx, ny, nz)
    op = tpmg.Operator.from_problem(p, nlevels=2)
    cx, cy, v = oracle.problem_coefficients(p)
    tpmg.set_variant(op.op, prec, 2, variant)
    u, f = rnd((nz, ny, nx), 70), rnd((nz, ny, nx), 71)
    out = torch.empty_like(dev(u, prec))
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    tpmg.smooth(op.op, 2, prec, 0.8, dev(u, prec), dev(f, prec), out, p.n, norm_out=nrm)
    ref = oracle.smooth(u, f, cx, cy, v, 0.8)
    assert rel(host(out), ref) < tol_inverse(prec, cx, cy, v), rel(host(out), ref)
    rnorm = np.linalg.norm(oracle.residual(u, f, cx, cy, v))
    assert abs(host(nrm)[0] - rnorm) / rnorm < max(TOL[prec], 1e-7)
    op.close()


def test_double_word_conversion_round_trip_is_exact():
    """FP64 -> double-word -> FP64 through an identity operator (omega^2 = 0, so A = I) reproduces
    float64(hi) + float64(lo) with hi = float32(x) and lo = float32(x - hi) bit for bit, over the
    float range (no infinities: the stencil's zero couplings would turn a neighbour's inf into NaN)
    including zeros, float denormals, the float extremes and round-to-nearest-even ties."""
    rng = np.random.default_rng(90)
    nz, ny, nx = 8, 4, 64
    n = nz * ny * nx
    vals = [rng.standard_normal(n // 2) * 10.0 ** rng.uniform(-30, 30, n // 2)]
    edge = [0.0, -0.0, 1.0, -1.0, 2.0 ** -60, 2.0 ** -61, 2.0 ** 100, 2.0 ** 101, 1e-300, 5e-324, 1e-40,
            3.4028234663852886e38 / 4, 1.1754943508222875e-38, 1 + 2.0 ** -24, 1 + 2.0 ** -23 + 2.0 ** -24,
            1 - 2.0 ** -25, 0.1, 1.0 / 3.0]
    # significands exactly halfway between two floats (ties to even) and just off it
    base = rng.uniform(1.0, 2.0, 64).astype(np.float32).astype(np.float64)
    ties = np.concatenate([base + 2.0 ** -24, base - 2.0 ** -24, base + 2.0 ** -24 * (1 + 2.0 ** -20)])
    x = np.concatenate([vals[0], np.array(edge), ties])
    x = np.concatenate([x, rng.standard_normal(n - x.size)]).reshape(nz, ny, nx)
    op = tpmg.Operator(nx, ny, nz, 0.0, 1.0 / nx, 1.0 / ny, 1.0 / nz, 1.0, 1)
    y = torch.empty(n, dtype=torch.float64, device="cuda")
    with np.errstate(under="ignore"):
        tpmg.apply_A(op.op, 1, tpmg.DW, torch.from_numpy(x.ravel()).cuda(), y, n)
        hi = x.ravel().astype(np.float32)
        lo = (x.ravel() - hi.astype(np.float64)).astype(np.float32)
        ref = hi.astype(np.float64) + lo.astype(np.float64)
    got = host(y)
    assert np.array_equal(got, ref), np.flatnonzero(got != ref)[:10]
    op.close()
