"""Pins of the oracle's exact constant-coefficient solver (oracle/spectral.py), no GPU needed.

It is checked against dense LU of the assembled operator on tiny grids (odd and even sizes, so the
half spectrum of the real transform and both parities of nx are covered), against the closed-form
eigenpairs (a single Fourier x DCT-II mode must come back divided by its eigenvalue, Sec. 2.1.1 and
Eq. (7)), and by the residual the (separately pinned) oracle operator leaves on a larger grid.
"""
import numpy as np
import pytest

import oracle
from helpers import assemble, fourier_dct_mode, mu_A, rel
from oracle import spectral


@pytest.mark.parametrize("shape", [(5, 6, 8), (3, 5, 7), (4, 4, 6), (1, 6, 5)])
def test_exact_solve_matches_dense_lu(shape):
    nz, ny, nx = shape
    cx, cy, v = 3.7, 1.3, 55.0
    A = assemble(lambda x: oracle.apply_A(x, cx, cy, np.full((ny, nx), v)), shape)
    f = np.random.default_rng(1).standard_normal(shape)
    u_lu = np.linalg.solve(A, f.ravel()).reshape(shape)
    u = spectral.exact_solve(f, cx, cy, v)
    assert rel(u, u_lu) < 1e-12


@pytest.mark.parametrize("p,q,m", [(0, 0, 0), (3, 2, 4), (5, 1, 1), (2, 5, 3)])
def test_exact_solve_divides_a_mode_by_its_eigenvalue(p, q, m):
    nx, ny, nz = 16, 12, 8
    cx, cy, v = 40.0, 25.0, 900.0
    x = fourier_dct_mode(nx, ny, nz, p, q, m, 0.3, -0.9)
    mu = float(mu_A(nx, ny, nz, cx, cy, v)[m, q, p])
    assert rel(spectral.exact_solve(x, cx, cy, v), x / mu) < 1e-13


def test_exact_solve_leaves_no_residual():
    """A 64 x 48 x 32 grid with the strong vertical coupling of the benchmark problems: the oracle's
    residual of the exact solution is at the level of rounding (kappa(A) ~ 1e5 times 1e-16)."""
    nx, ny, nz = 64, 48, 32
    cx, cy, v = 1e-2 * 64 ** 2, 1e-2 * 48 ** 2, 1e-2 * 1e3 * 32 ** 2
    f = np.random.default_rng(2).uniform(-1, 1, (nz, ny, nx))
    u = spectral.exact_solve(f, cx, cy, v)
    r = oracle.residual(u, f, cx, cy, np.full((ny, nx), v))
    assert np.linalg.norm(r) / np.linalg.norm(f) < 1e-12


def test_thread_count_does_not_change_the_oracle():
    """The oracle's loops over cells and columns may run on several host threads; each cell is
    computed by the same code whichever thread takes it and the norms run in index order, so a
    multigrid solve gives the same iterate and history bit for bit on 1 and on 4 threads."""
    nx, ny, nz = 32, 32, 16
    rng = np.random.default_rng(3)
    v = 1e-2 * 1e3 * nz ** 2 * (1.0 + 0.5 * rng.random((ny, nx)))
    f = rng.standard_normal((nz, ny, nx))
    cx = cy = 1e-2 * nx ** 2
    before = oracle.set_threads(0)
    try:
        oracle.set_threads(1)
        u1, it1, h1, _ = oracle.mg_solve(f, cx, cy, v, 3, tol=1e-8)
        oracle.set_threads(4)
        u4, it4, h4, _ = oracle.mg_solve(f, cx, cy, v, 3, tol=1e-8)
    finally:
        oracle.set_threads(before)
    assert it1 == it4
    assert np.array_equal(u1, u4) and np.array_equal(np.asarray(h1), np.asarray(h4))
