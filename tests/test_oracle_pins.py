"""Pins of the oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the passage it follows. None of them re-types the oracle's formula: they use
closed-form eigenpairs, library FFT/DCT solves, dense linear algebra on tiny grids, values the
paper prints (tests/golden/) and invariants (symmetry, positive definiteness, fixed points,
reproduction of linear functions).
"""
import numpy as np
import pytest
import scipy.linalg

import oracle
from helpers import (assemble, cg_iteration_bound, fourier_dct_mode, mu_A, mu_M, read_golden,
                     rel, spectral_solve)

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

# deliberately unequal sizes and coefficients so that a transposed index or a swapped cx/cy fails
NX, NY, NZ = 8, 6, 5
CX, CY, V = 3.7, 1.3, 55.0


def rand_field(shape, seed):
    return np.random.default_rng(seed).standard_normal(shape)


def rand_v(ny, nx, seed):
    return 10.0 + 90.0 * np.random.default_rng(seed).random((ny, nx))


# ---------------------------------------------------------------- operator A (Sec. 2.1.1, Eq. 6)

@pytest.mark.parametrize("p,q,m", [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (3, 2, 4),
                                   (4, 3, 2), (2, 5, 3), (7, 1, 1)])
@pytest.mark.parametrize("phase", [0.0, 0.7])
def test_apply_A_fourier_dct_eigenpairs(p, q, m, phase):
    """Constant coefficients: A is diagonal in Fourier(x) x Fourier(y) x DCT-II(z) with
    eigenvalue 1 + 4cx sin^2(pi p/nx) + 4cy sin^2(pi q/ny) + 4v sin^2(pi m/(2nz))."""
    x = fourier_dct_mode(NX, NY, NZ, p, q, m, phase, -phase)
    y = oracle.apply_A(x, CX, CY, V)
    mu = mu_A(NX, NY, NZ, CX, CY, V)[m, q, p]
    assert rel(y, mu * x) < 1e-13


def test_apply_A_constant_vector_is_fixed():
    """A 1 = 1: horizontal and vertical couplings of a constant field cancel (Neumann ends)."""
    v = rand_v(NY, NX, 1)
    y = oracle.apply_A(np.ones((NZ, NY, NX)), CX, CY, v)
    assert np.max(np.abs(y - 1.0)) < 1e-12


def test_apply_A_vertical_part_indexes_v_by_column():
    """x = g_ij h_k with h a DCT-II mode: (A x - x) splits into a horizontal part that is
    independent of v and a vertical part v_ij 4 sin^2(pi m/2nz) g_ij h_k."""
    v = rand_v(NY, NX, 2)
    m = 3
    k = np.arange(NZ)[:, None, None]
    h = np.cos(np.pi * m * (k + 0.5) / NZ)
    # horizontally constant: only the vertical part remains
    x = h * np.ones((1, NY, NX))
    lam_z = 4 * np.sin(np.pi * m / (2 * NZ)) ** 2
    assert rel(oracle.apply_A(x, CX, CY, v) - x, v[None] * lam_z * x) < 1e-13
    # vertically constant: the result does not depend on v at all
    g = rand_field((1, NY, NX), 3) * np.ones((NZ, 1, 1))
    y1 = oracle.apply_A(g, CX, CY, v)
    y2 = oracle.apply_A(g, CX, CY, rand_v(NY, NX, 4))
    assert rel(y1, y2) < 1e-13


def test_flatbox_entries_match_paper():
    """Sec. 2.1.1 prints the flat-box matrix entries; assemble A on a tiny grid and read them."""
    g = read_golden("flatbox_entries.txt")
    cx = cy = g["omega2"] / g["h"] ** 2
    v = g["omega2"] * g["lambda2"] / g["hz"] ** 2
    nx, ny, nz = 4, 4, 4
    A = assemble(lambda x: oracle.apply_A(x, cx, cy, v), (nz, ny, nx))

    def lin(i, j, k):
        return (k * ny + j) * nx + i

    c = lin(1, 2, 2)
    assert A[c, c] == pytest.approx(g["interior_diag"], rel=1e-14)
    assert A[c, lin(2, 2, 2)] == pytest.approx(g["horizontal_offdiag"], rel=1e-14)
    assert A[c, lin(1, 1, 2)] == pytest.approx(g["horizontal_offdiag"], rel=1e-14)
    assert A[c, lin(1, 2, 1)] == pytest.approx(g["vertical_offdiag"], rel=1e-14)
    assert A[c, lin(1, 2, 3)] == pytest.approx(g["vertical_offdiag"], rel=1e-14)
    e = lin(1, 2, 0)
    assert A[e, e] == pytest.approx(g["neumann_end_diag"], rel=1e-14)
    # seven-point stencil: at most 7 non-zeros per row
    assert np.max(np.count_nonzero(A, axis=1)) == 7


def test_dense_A_spectrum_constant_coefficients():
    """Eigenvalues of the assembled A equal the closed-form set, with multiplicity."""
    nx, ny, nz = 4, 6, 3
    A = assemble(lambda x: oracle.apply_A(x, CX, CY, V), (nz, ny, nx))
    assert np.array_equal(A, A.T)
    ev = np.sort(np.linalg.eigvalsh(A))
    ref = np.sort(mu_A(nx, ny, nz, CX, CY, V).ravel())
    assert np.max(np.abs(ev - ref)) / ref.max() < 1e-13


def test_dense_A_symmetric_positive_definite_variable_v():
    """A = I + (positive semi-definite couplings): symmetric, Cholesky succeeds, lambda_min = 1."""
    nx, ny, nz = 4, 6, 3
    v = rand_v(ny, nx, 5)
    A = assemble(lambda x: oracle.apply_A(x, CX, CY, v), (nz, ny, nx))
    assert np.array_equal(A, A.T)
    np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() == pytest.approx(1.0, abs=1e-10)


# ---------------------------------------------------------------- line solve M^{-1} (Sec. 2.2)

def test_line_solve_inverts_the_column_blocks_of_A():
    """M is the block-diagonal (per column) part of A; compare with dense LU per column."""
    nx, ny, nz = 4, 3, 7
    v = rand_v(ny, nx, 6)
    A = assemble(lambda x: oracle.apply_A(x, CX, CY, v), (nz, ny, nx))
    b = rand_field((nz, ny, nx), 7)
    x = oracle.line_solve(b, CX, CY, v)
    for j in range(ny):
        for i in range(nx):
            rows = [(k * ny + j) * nx + i for k in range(nz)]
            Mblk = A[np.ix_(rows, rows)]
            ref = scipy.linalg.lu_solve(scipy.linalg.lu_factor(Mblk), b[:, j, i])
            assert rel(x[:, j, i], ref) < 1e-13


@pytest.mark.parametrize("m", [0, 1, 4])
def test_line_solve_dct_eigen(m):
    """M^{-1}(g_ij h_k) = g_ij h_k / (1 + 2cx + 2cy + 4 v_ij sin^2(pi m/2nz)) for a DCT-II mode h."""
    v = rand_v(NY, NX, 8)
    k = np.arange(NZ)[:, None, None]
    g = rand_field((1, NY, NX), 9)
    x = g * np.cos(np.pi * m * (k + 0.5) / NZ)
    mu = 1 + 2 * CX + 2 * CY + 4 * v[None] * np.sin(np.pi * m / (2 * NZ)) ** 2
    assert rel(oracle.line_solve(x, CX, CY, v), x / mu) < 1e-13


def test_line_solve_single_level_column():
    """nz = 1: M is the diagonal 1 + 2cx + 2cy (no vertical neighbours)."""
    b = rand_field((1, NY, NX), 10)
    assert rel(oracle.line_solve(b, CX, CY, 5.0), b / (1 + 2 * CX + 2 * CY)) < 1e-15


# ---------------------------------------------------------------- smoother / residual (Eq. 11)

@pytest.mark.parametrize("p,q,m", [(0, 0, 0), (4, 3, 0), (1, 2, 3), (3, 0, 4)])
def test_smoother_error_propagation_on_modes(p, q, m):
    """With f = 0 the error e = u evolves as (1 - rho mu_A/mu_M) e on every eigenmode."""
    rho = 0.8
    x = fourier_dct_mode(NX, NY, NZ, p, q, m)
    out = oracle.smooth(x, np.zeros_like(x), CX, CY, V, rho)
    factor = 1 - rho * mu_A(NX, NY, NZ, CX, CY, V)[m, q, p] / mu_M(NX, NY, NZ, CX, CY, V)[m, q, p]
    assert rel(out, factor * x) < 1e-12


def test_smoother_and_residual_fixed_point():
    """u* with f = A u* is a fixed point of the smoother and has zero residual."""
    v = rand_v(NY, NX, 11)
    u = rand_field((NZ, NY, NX), 12)
    f = oracle.apply_A(u, CX, CY, v)
    assert rel(oracle.smooth(u, f, CX, CY, v, 0.8), u) < 1e-13
    assert np.max(np.abs(oracle.residual(u, f, CX, CY, v))) < 1e-10 * np.max(np.abs(f))


@pytest.mark.parametrize("p,q,m", [(2, 1, 1), (0, 3, 2)])
def test_residual_on_mode(p, q, m):
    x = fourier_dct_mode(NX, NY, NZ, p, q, m)
    r = oracle.residual(x, np.zeros_like(x), CX, CY, V)
    assert rel(r, -mu_A(NX, NY, NZ, CX, CY, V)[m, q, p] * x) < 1e-13


# ---------------------------------------------------------------- transfers (Sec. 2.2)

def test_restriction_reproduces_bilinear_functions():
    """The cell average of a separable bilinear function equals its value at the coarse centre."""
    nxf, nyf, nz = 8, 12, 3
    xf = (np.arange(nxf) + 0.5) / nxf
    yf = (np.arange(nyf) + 0.5) / nyf
    g = np.array([1.0, -2.0, 0.5])[:, None, None]
    rf = g * ((0.3 + 1.7 * xf)[None, None, :] * (2.0 - 0.9 * yf)[None, :, None])
    xc = (np.arange(nxf // 2) + 0.5) / (nxf // 2)
    yc = (np.arange(nyf // 2) + 0.5) / (nyf // 2)
    ref = g * ((0.3 + 1.7 * xc)[None, None, :] * (2.0 - 0.9 * yc)[None, :, None])
    assert rel(oracle.restrict(rf), ref) < 1e-14


def test_restriction_weights():
    """Each coarse value is 1/4 of the sum of exactly its 2x2 children."""
    rf = np.zeros((1, 4, 6))
    rf[0, 2, 3] = 1.0  # child (i=3, j=2) belongs to coarse (I=1, J=1)
    fc = oracle.restrict(rf)
    ref = np.zeros((1, 2, 3))
    ref[0, 1, 1] = 0.25
    assert np.array_equal(fc, ref)


def test_prolongation_reproduces_bilinear_functions_away_from_the_seam():
    """Linear interpolation of cell-centred data reproduces a bilinear function at fine cells
    whose two interpolation neighbours do not wrap around the periodic boundary."""
    nxc, nyc, nz = 6, 5, 2
    Xc = (np.arange(nxc) + 0.5) / nxc
    Yc = (np.arange(nyc) + 0.5) / nyc
    fx = lambda x: 0.4 - 2.5 * x
    fy = lambda y: 1.0 + 3.0 * y
    uc = np.ones((nz, 1, 1)) * (fx(Xc)[None, None, :] * fy(Yc)[None, :, None])
    out = oracle.prolongate_add(uc, np.zeros((nz, 2 * nyc, 2 * nxc)))
    xf = (np.arange(2 * nxc) + 0.5) / (2 * nxc)
    yf = (np.arange(2 * nyc) + 0.5) / (2 * nyc)
    ref = np.ones((nz, 1, 1)) * (fx(xf)[None, None, :] * fy(yf)[None, :, None])
    inner = (slice(None), slice(1, 2 * nyc - 1), slice(1, 2 * nxc - 1))
    assert rel(out[inner], ref[inner]) < 1e-14


def test_prolongation_of_constant_and_accumulation():
    uc = np.full((3, 3, 4), 2.5)
    base = np.random.default_rng(13).standard_normal((3, 6, 8))
    out = oracle.prolongate_add(uc, base)
    assert np.max(np.abs(out - base - 2.5)) < 1e-14


def test_coarse_vertical_coefficient_is_child_average():
    vf = np.arange(24, dtype=float).reshape(4, 6)
    vc = oracle.coarsen_v(vf)
    assert vc[1, 2] == pytest.approx((vf[2, 4] + vf[2, 5] + vf[3, 4] + vf[3, 5]) / 4)


# ---------------------------------------------------------------- solvers (Sec. 2.2, Alg. 1)

def _const_problem(nx=32, ny=16, nz=8, seed=14):
    # coarsest level of a 3-level hierarchy has cx = 0.25, cy ~ 0.16: well conditioned, so two
    # smoothing steps solve it (Sec. 2.2, last paragraph; Sec. 5.2 for what happens otherwise)
    cx, cy, v = 4.0, 2.5, 900.0
    f = rand_field((nz, ny, nx), seed)
    return f, cx, cy, v


def test_mg_solve_converges_to_spectral_solution():
    """Constant coefficients: repeated V(2,2) cycles reach the exact FFT/DCT solution."""
    f, cx, cy, v = _const_problem()
    u, it, hist, conv = oracle.mg_solve(f, cx, cy, v, nlevels=3, tol=1e-12, max_iter=60)
    assert conv
    assert rel(u, spectral_solve(f, cx, cy, v)) < 1e-10


def test_mg_vcycle_contraction_band():
    """On the paper-shaped problem (omega = 4.2 h, Eq. (4); kappa ~ 142) the tensor-product
    multigrid contracts the residual at least as fast as the paper's V(1,1) cycles, about
    10^(-5/8) ~ 0.24 per cycle (Table SingleGPUTiming, 8-9 cycles for 5 orders); V(2,2) must do
    at least that well. With more coarse smoothing steps it can only improve (Sec. 5.2)."""
    # 4 levels from 64: coarsest c = 17.64/64 ~ 0.28, comparable to the paper's 5-level setup
    nx, nz = 64, 16
    c = 4.2 ** 2
    v = 1e-2 * 1e3 * nz ** 2
    f = rand_field((nz, nx, nx), 15)
    u, it, hist, conv = oracle.mg_solve(f, c, c, v, nlevels=4, tol=1e-8, max_iter=40)
    assert conv
    rates = hist[1:] / hist[:-1]
    assert np.max(rates[1:]) < 0.24
    _, it20, _, _ = oracle.mg_solve(f, c, c, v, nlevels=4, tol=1e-8, max_iter=40, n_coarse=20)
    assert it20 <= it


def test_mg_and_cg_match_dense_lu_variable_v():
    """Variable lambda^2: multigrid, CG and iterative refinement reach the dense LU solution on a
    tiny grid."""
    nx, ny, nz = 8, 8, 4
    cx, cy = 30.0, 30.0
    v = rand_v(ny, nx, 16) * 10
    f = rand_field((nz, ny, nx), 17)
    A = assemble(lambda x: oracle.apply_A(x, cx, cy, v), (nz, ny, nx))
    ref = np.linalg.solve(A, f.ravel()).reshape(f.shape)
    u_mg, _, _, c1 = oracle.mg_solve(f, cx, cy, v, nlevels=3, tol=1e-13, max_iter=200)
    u_cg, _, _, c2 = oracle.cg_solve(f, cx, cy, v, tol=1e-13, max_iter=500)
    u_ir, _, _, c3 = oracle.ir_solve(f, cx, cy, v, nlevels=3, tol=1e-13, max_iter=200)
    assert c1 and c2 and c3
    assert rel(u_mg, ref) < 1e-10
    assert rel(u_cg, ref) < 1e-10
    assert rel(u_ir, ref) < 1e-10


def test_preconditioned_condition_number_matches_paper():
    """Sec. 2.1.1, Eq. (7): kappa(M^{-1} A) = 1 + 8 omega^2/h^2; with omega = 4.2 h the paper
    states kappa ~ 142. Generalised eigenvalues of the assembled (A, M) on a tiny grid."""
    g = read_golden("condition_number.txt")
    c = g["omega_over_h"] ** 2
    nx, ny, nz = 4, 4, 3
    v = 500.0
    A = assemble(lambda x: oracle.apply_A(x, c, c, v), (nz, ny, nx))
    Minv = assemble(lambda x: oracle.line_solve(x, c, c, v), (nz, ny, nx))
    ev = np.linalg.eigvals(Minv @ A).real
    kappa = ev.max() / ev.min()
    assert kappa == pytest.approx(g["kappa_exact"], rel=1e-10)
    assert round(kappa) == g["kappa_paper_rounded"]


def test_cg_iterations_within_classical_bound():
    """CG on the paper-shaped problem (kappa = 142.12) needs no more than
    ceil(sqrt(kappa)/2 ln(2/eps)) iterations, and reaches the spectral solution."""
    nx, nz = 16, 8
    c = 4.2 ** 2
    v = 1e-2 * 1e3 * nz ** 2
    f = rand_field((nz, nx, nx), 18)
    tol = 1e-6
    u, it, hist, conv = oracle.cg_solve(f, c, c, v, tol=tol, max_iter=1000)
    assert conv
    assert it <= cg_iteration_bound(1 + 8 * c, tol)
    # the residual reduction bounds the error by kappa(A) * tol in the 2-norm
    assert rel(u, spectral_solve(f, c, c, v)) < 1e-6 * (1 + 8 * c + 4 * v)


def test_iterative_refinement_reproduces_the_multigrid_iteration():
    """The V-cycle is a linear iteration, so one V-cycle on the correction equation from a zero
    guess gives exactly the next multigrid iterate: IR and MG histories agree."""
    nx, nz = 16, 8
    cx = cy = 1e-2 * nx ** 2
    v = 1e-2 * 1e3 * nz ** 2
    f = rand_field((nz, nx, nx), 19)
    _, it1, h1, _ = oracle.mg_solve(f, cx, cy, v, nlevels=2, tol=1e-10, max_iter=30)
    _, it2, h2, _ = oracle.ir_solve(f, cx, cy, v, nlevels=2, tol=1e-10, max_iter=30)
    assert it1 == it2
    assert np.allclose(h1, h2, rtol=1e-6, atol=1e-14)


def test_single_level_cycle_is_plain_smoothing():
    """With one level the cycle is n_coarse smoothing steps (no coarse grid)."""
    f, cx, cy, v = _const_problem(8, 8, 4)
    u0 = rand_field(f.shape, 20)
    u = oracle.vcycle(u0, f, cx, cy, v, nlevels=1, n_coarse=2, rho=0.8)
    ref = oracle.smooth(oracle.smooth(u0, f, cx, cy, v, 0.8), f, cx, cy, v, 0.8)
    assert rel(u, ref) < 1e-15


def test_zero_rhs_is_converged_immediately():
    z = np.zeros((4, 8, 8))
    u, it, hist, conv = oracle.mg_solve(z, 1.0, 1.0, 1.0, nlevels=2)
    assert conv and it == 0 and not u.any()


def _dense_vcycle_map(nx, ny, nz, L, cx, cy, v, nu_pre, nu_post, n_coarse, rho):
    """Algorithm 1 written in matrix form on a tiny grid. For level l, B_l maps a right-hand side
    to the cycle's approximation starting from zero; the fine cycle from u is
    u_new = S^nu_post [S^nu_pre u + (I - S^nu_pre) A^-1 f + P B_{L-1} R r] + (I - S^nu_post) A^-1 f.
    Smoother S = I - rho M^-1 A (Eq. 11); the coarsest level does n_coarse smoothing steps from
    zero, i.e. B_1 = (I - S_1^n_coarse) A_1^-1. Coarse operators are rediscretised with cx/4,
    cy/4 and the 2x2-averaged v per level."""
    ops = {}
    vl, cxl, cyl, nxl, nyl = np.asarray(v, float), cx, cy, nx, ny
    for l in range(L, 0, -1):
        shape = (nz, nyl, nxl)
        A = assemble(lambda x, a=cxl, b=cyl, c=vl: oracle.apply_A(x, a, b, c), shape)
        Minv = assemble(lambda x, a=cxl, b=cyl, c=vl: oracle.line_solve(x, a, b, c), shape)
        ops[l] = dict(A=A, S=np.eye(A.shape[0]) - rho * Minv @ A, Ainv=np.linalg.inv(A), shape=shape)
        if l > 1:
            ops[l]["R"] = assemble(oracle.restrict, shape)
            ops[l]["P"] = assemble(lambda x, s=shape: oracle.prolongate_add(
                x, np.zeros(s)), (nz, nyl // 2, nxl // 2))
            vl = vl.reshape(nyl // 2, 2, nxl // 2, 2).mean(axis=(1, 3))
            cxl, cyl, nxl, nyl = cxl / 4, cyl / 4, nxl // 2, nyl // 2
    mp = np.linalg.matrix_power

    def B(l):
        o = ops[l]
        n = o["A"].shape[0]
        if l == 1:
            return (np.eye(n) - mp(o["S"], n_coarse)) @ o["Ainv"]
        pre = (np.eye(n) - mp(o["S"], nu_pre)) @ o["Ainv"]
        x = pre + o["P"] @ B(l - 1) @ o["R"] @ (np.eye(n) - o["A"] @ pre)
        return mp(o["S"], nu_post) @ x + (np.eye(n) - mp(o["S"], nu_post)) @ o["Ainv"]

    o = ops[L]
    n = o["A"].shape[0]
    Bc = B(L - 1)

    def cycle(u, f):
        u, f = u.ravel(), f.ravel()
        x = mp(o["S"], nu_pre) @ u + (np.eye(n) - mp(o["S"], nu_pre)) @ o["Ainv"] @ f
        x = x + o["P"] @ Bc @ o["R"] @ (f - o["A"] @ x)
        return (mp(o["S"], nu_post) @ x + (np.eye(n) - mp(o["S"], nu_post)) @ o["Ainv"] @ f).reshape(o["shape"])

    return cycle


@pytest.mark.parametrize("nu_pre,nu_post,n_coarse,rho", [(2, 2, 2, 0.8), (1, 1, 2, 2 / 3), (1, 3, 3, 0.7)])
def test_vcycle_matches_matrix_form_of_algorithm_1(nu_pre, nu_post, n_coarse, rho):
    """One oracle V-cycle equals Algorithm 1's error-propagation form built from dense matrices
    (3 levels, variable lambda^2, unequal cx and cy)."""
    nx, ny, nz, L = 8, 8, 3, 3
    cx, cy = 6.0, 2.0
    v = rand_v(ny, nx, 21)
    u0 = rand_field((nz, ny, nx), 22)
    f = rand_field((nz, ny, nx), 23)
    cyc = _dense_vcycle_map(nx, ny, nz, L, cx, cy, v, nu_pre, nu_post, n_coarse, rho)
    got = oracle.vcycle(u0, f, cx, cy, v, nlevels=L, nu_pre=nu_pre, nu_post=nu_post,
                        n_coarse=n_coarse, rho=rho)
    assert rel(got, cyc(u0, f)) < 1e-11


def test_paper_shaped_iteration_counts_near_the_paper():
    """Sec. 5.1, Table SingleGPUTiming: with omega = 4.2 h, 5 levels, V(1,1), rho = 2/3 and eps =
    1e-5 the paper's multigrid takes 8-9 cycles and line-preconditioned CG 58-70 iterations. The
    paper's lambda(h) is not reproduced in its text (this build takes lambda^2 = 1e3) and the grid
    here is 128^2 x 64, so the counts are pinned to a band: multigrid within two cycles of the
    paper's 9 at nx = 128, CG no more than the classical bound ceil(sqrt(kappa)/2 ln(2/eps)) and
    no fewer than 3/4 of the paper's smallest count."""
    from paper_1402_3545_gb300 import workloads
    g = read_golden("paper_iterations.txt")
    p = workloads.paper_shaped(128, 64)
    assert p.nlevels == 5
    cx, cy, v = oracle.problem_coefficients(p)
    f = p.rhs()
    _, it_mg, _, conv_mg = oracle.mg_solve(f, cx, cy, v, p.nlevels, tol=1e-5, max_iter=50, nu_pre=1, nu_post=1,
                                           rho=2.0 / 3.0)
    assert conv_mg and abs(it_mg - g["mg_128"]) <= 2, it_mg
    _, it_cg, _, conv_cg = oracle.cg_solve(f, cx, cy, v, tol=1e-5, max_iter=500)
    assert conv_cg
    assert 0.75 * g["cg_768"] <= it_cg <= cg_iteration_bound(1 + 8 * cx, 1e-5), it_cg
