"""Pins of the panel oracle (oracle/panel.py, oracle/panel_oracle.c): the paper's own operator, Eq. (1)
on one gnomonic cubed-sphere panel in the factorised form of Eq. (14) (Sec. 2.1.1, Sec. 3.1). No GPU.

What fixes it independently of its own code: the panel's exact area (a sixth of the sphere) and the
length of its boundary (four great-circle arcs of arccos(1/3)); the radial shell volume; symmetry and
positive definiteness of the assembled operator; the flat limit -- on a tiny patch at the panel
centre with a thin shell the spectrum must approach the closed form of the Dirichlet x Dirichlet x
Neumann box, which fails for a wrong sign, a wrong boundary treatment or a transposed index; the line
solve against dense LU of each column block; the transfers' matrices against their stated weights;
multigrid and CG against dense LU.
"""
import numpy as np
import pytest

from helpers import assemble, rel
from oracle import panel


def test_panel_area_is_a_sixth_of_the_sphere_and_levels_add_up():
    P = panel.PanelProblem(64, 48, 4, 4, 1e-2, 1.0, 1.6e-3)
    assert abs(P.levels[4]["area"].sum() - 4.0 * np.pi / 6.0) < 1e-13
    for l in (3, 2, 1):  # a coarse cell is the union of its 2 x 2 children
        fine = P.levels[l + 1]["area"]
        ch = fine[0::2, 0::2] + fine[1::2, 0::2] + fine[0::2, 1::2] + fine[1::2, 1::2]
        assert np.max(np.abs(P.levels[l]["area"] - ch)) < 1e-15


def test_panel_boundary_length():
    """Each edge of a cube face is the great-circle arc between (1, -1, 1)/sqrt(3) and
    (1, 1, 1)/sqrt(3), of length arccos(1/3); the boundary faces of the grid tile the four edges."""
    om2 = 1.0
    for nx, ny in [(8, 8), (10, 6)]:
        xs = -1.0 + 2.0 * np.arange(nx + 1) / nx
        ys = -1.0 + 2.0 * np.arange(ny + 1) / ny
        left = panel.arc(panel.sphere_point(-1.0, ys[:-1]), panel.sphere_point(-1.0, ys[1:])).sum()
        bottom = panel.arc(panel.sphere_point(xs[:-1], -1.0), panel.sphere_point(xs[1:], -1.0)).sum()
        assert abs(left - np.arccos(1.0 / 3.0)) < 1e-14 and abs(bottom - np.arccos(1.0 / 3.0)) < 1e-14
        g = panel.panel_geometry(nx, ny, om2)
        assert g["ax"].shape == (ny, nx + 1) and g["ay"].shape == (ny + 1, nx)
        assert np.all(g["ax"] < 0) and np.all(g["ay"] < 0)


def test_radial_mass_is_the_shell_volume_and_stiffness_is_symmetric():
    nz, H, om2, lam2 = 16, 0.05, 0.3, 2.0
    a, b, c = panel.radial_vectors(nz, H, om2, lam2)
    hz = H / nz
    assert abs(np.sum(a) * hz - ((1 + H) ** 3 - 1) / 3.0) < 1e-15
    assert b[0] == 0.0 and c[-1] == 0.0
    assert np.allclose(c[:-1], b[1:], rtol=0, atol=0)  # the coupling of k and k+1 is one face's


@pytest.mark.parametrize("shape", [(4, 5, 6), (3, 6, 4)])
def test_operator_is_symmetric_positive_definite(shape):
    nz, ny, nx = shape
    P = panel.PanelProblem(nx, ny, nz, 1, (4.2 * np.pi / (2 * nx)) ** 2, 1.0, 0.01)
    A = assemble(P.apply_A, shape)
    assert np.max(np.abs(A - A.T)) < 1e-14 * np.max(np.abs(A))
    np.linalg.cholesky(A)
    assert np.min(np.linalg.eigvalsh(A)) > 0


def test_flat_limit_spectrum():
    """extent 1e-3 (an nx x ny patch of h x hy cells at the panel centre, distortion O(extent^2)) and
    H = 1e-9 (r = 1 throughout): A has the eigenvalues of the flat box in integrated form,
    h hy + omega^2 (hy / h) 4 sin^2(pi p / (2 (nx + 1))) + omega^2 (h / hy) 4 sin^2(pi q / (2 (ny + 1)))
      + h hy (omega^2 lambda^2 / h_z^2) 4 sin^2(pi m / (2 nz)),   p = 1..nx, q = 1..ny, m = 0..nz-1
    (Dirichlet with the ghost value 0 one cell out; Neumann with the mirror ghost)."""
    nx, ny, nz, ext, H = 6, 5, 4, 1e-3, 1e-9
    h = 2 * ext / nx
    hy = 2 * ext / ny
    # lambda^2 scaled so the vertical coupling is of the horizontal one's size: the spectrum then
    # spans a few decades and a dense eigensolver resolves every eigenvalue to ~1e-12
    om2, lam2 = (3.0 * h) ** 2, 0.7 * (H / nz) ** 2 / h ** 2
    P = panel.PanelProblem(nx, ny, nz, 1, om2, lam2, H, extent=ext)
    A = assemble(P.apply_A, (nz, ny, nx))
    got = np.sort(np.linalg.eigvalsh(A))
    p = np.arange(1, nx + 1)[:, None, None]
    q = np.arange(1, ny + 1)[None, :, None]
    m = np.arange(nz)[None, None, :]
    hz = H / nz
    # cells are h x hy rectangles: |T| = h hy, x-faces |e| / d = hy / h, y-faces h / hy
    lam = (h * hy + om2 * (hy / h) * 4 * np.sin(np.pi * p / (2 * (nx + 1))) ** 2
           + om2 * (h / hy) * 4 * np.sin(np.pi * q / (2 * (ny + 1))) ** 2
           + h * hy * om2 * lam2 / hz ** 2 * 4 * np.sin(np.pi * m / (2 * nz)) ** 2)
    want = np.sort(lam.ravel())
    assert np.max(np.abs(got - want) / want) < 1e-5


def test_line_solve_is_the_column_blocks_inverse():
    nx, ny, nz = 5, 4, 7
    P = panel.PanelProblem(nx, ny, nz, 1, 0.02, 1.3, 0.02)
    A = assemble(P.apply_A, (nz, ny, nx))
    r = np.random.default_rng(3).standard_normal((nz, ny, nx))
    x = P.line_solve(r)
    for j in range(ny):
        for i in range(nx):
            idx = [(k * ny + j) * nx + i for k in range(nz)]
            blk = A[np.ix_(idx, idx)]
            assert rel(x[:, j, i], np.linalg.solve(blk, r[:, j, i])) < 1e-13


def test_transfer_matrices_have_the_stated_weights():
    nz, nyc, nxc = 1, 3, 4
    R = assemble(panel.restrict, (nz, 2 * nyc, 2 * nxc))
    for I in range(nxc):
        for J in range(nyc):
            row = R[J * nxc + I].reshape(2 * nyc, 2 * nxc)
            want = np.zeros((2 * nyc, 2 * nxc))
            want[2 * J:2 * J + 2, 2 * I:2 * I + 2] = 1.0
            assert np.array_equal(row, want)
    Pm = assemble(lambda uc: panel.prolongate_add(uc, np.zeros((nz, 2 * nyc, 2 * nxc))), (nz, nyc, nxc))
    ones = Pm @ np.ones(nxc * nyc)
    fine = ones.reshape(2 * nyc, 2 * nxc)
    assert np.allclose(fine[1:-1, 1:-1], 1.0)  # interior: the weights 9/16, 3/16, 3/16, 1/16 add to 1
    assert np.allclose(fine[0, 1:-1], 0.75) and np.allclose(fine[1:-1, 0], 0.75)  # one ghost direction
    assert np.isclose(fine[0, 0], 0.5625)  # corner: only the 9/16 weight stays on the panel


@pytest.mark.parametrize("solver", ["mg", "cg"])
def test_solvers_against_dense_lu(solver):
    nx, ny, nz = 8, 8, 4
    P = panel.PanelProblem(nx, ny, nz, 3, (4.2 * np.pi / (2 * nx)) ** 2, 1.0, 0.01)
    A = assemble(P.apply_A, (nz, ny, nx))
    f = np.random.default_rng(5).standard_normal((nz, ny, nx))
    u_lu = np.linalg.solve(A, f.ravel())
    if solver == "mg":
        u, it, hist, conv = P.mg_solve(f, tol=1e-12, max_iter=80, nu_pre=1, nu_post=1, rho=2.0 / 3.0)
    else:
        u, it, hist, conv = P.cg_solve(f, tol=1e-12, max_iter=500)
    assert conv
    assert rel(u.ravel(), u_lu) < 1e-10
