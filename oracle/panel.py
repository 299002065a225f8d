"""Oracle of the paper's own operator on one cubed-sphere panel (test infrastructure).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
module; the CUDA library computes its own geometry and shares no code with it.

The model equation, Eq. (1), -omega^2 (Lap_S u + lambda^2 r^-2 d_r (r^2 d_r u)) + u = f on one panel
of the sphere times r in [1, 1 + H], discretised by cell-centred finite volumes (Sec. 2.1.1) on a
gnomonic cubed-sphere panel (equidistant in the cube-face coordinates X, Y in [-1, 1]; a point maps
to (X, Y, 1) / sqrt(1 + X^2 + Y^2) on the unit sphere), homogeneous Dirichlet on the panel boundary
and Neumann at r = 1 and r = 1 + H. Integrating over cell T x [r_{k-1/2}, r_{k+1/2}] and dividing by
the vertical spacing h_z = H / nz gives the factorised stencil of Eq. (14):

- |T|: the cell's area on the unit sphere, exactly (the integral of (1 + X^2 + Y^2)^(-3/2) over the
  cell, whose antiderivative is atan(X Y / sqrt(1 + X^2 + Y^2)));
- alpha_{TT'} = -omega^2 |e_{TT'}| / d_{TT'}: the two-point flux through the shared edge, |e| its
  great-circle length (the gnomonic grid lines are great circles), d the great-circle distance of
  the two cell centres (the images of the cells' coordinate midpoints); a boundary face couples to
  the ghost cell of the extended grid, whose value is 0;
- a_k = (r_{k+1/2}^3 - r_{k-1/2}^3) / (3 h_z) (the radial mass), b_k = -omega^2 lambda^2
  r_{k-1/2}^2 / h_z^2 (0 at k = 0) and c_k = -omega^2 lambda^2 r_{k+1/2}^2 / h_z^2 (0 at k = nz-1)
  (the radial stiffness), d_k = 1.

Coarse multigrid levels rediscretise the same panel with half the cells per direction (the paper's
coefficients "depend on the multigrid level", Sec. 3.1). The arithmetic of the operator, the line
solve, the transfers, the V-cycle and CG is in ``panel_oracle.c``.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _f64, _load, _ptr

_I, _D, _P = ctypes.c_int, ctypes.c_double, ctypes.c_void_p


def _lib():
    lib = _load()
    if not getattr(lib, "_panel_ready", False):
        geo = [_P, _P, _P, _P, _P, _P]
        for name, args, res in [
            ("orc_panel_apply_A", [_I, _I, _I] + geo + [_P, _P], None),
            ("orc_panel_line_solve", [_I, _I, _I] + geo + [_P, _P], None),
            ("orc_panel_restrict", [_I, _I, _I, _P, _P], None),
            ("orc_panel_prolongate_add", [_I, _I, _I, _P, _P], None),
            ("orc_panel_mg_solve", [_I, _P, _P, _I, _P, _P, _P, _P, _P, _P, _I, _I, _I, _D, _D, _I, _P, _P, _P, _P], _I),
            ("orc_panel_cg_solve", [_I, _I, _I] + geo + [_D, _I, _P, _P, _P, _P], _I),
        ]:
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        lib._panel_ready = True
    return lib


def sphere_point(X, Y):
    """Image of the cube-face point (X, Y, 1) on the unit sphere; X, Y broadcast."""
    X, Y = np.broadcast_arrays(np.asarray(X, dtype=np.float64), np.asarray(Y, dtype=np.float64))
    rho = np.sqrt(1.0 + X * X + Y * Y)
    return np.stack([X / rho, Y / rho, 1.0 / rho], axis=-1)


def arc(p, q):
    """Great-circle distance of unit vectors p and q (atan2 form: accurate for short arcs)."""
    return np.arctan2(np.linalg.norm(np.cross(p, q), axis=-1), np.sum(p * q, axis=-1))


def _area_antiderivative(X, Y):
    return np.arctan(X * Y / np.sqrt(1.0 + X * X + Y * Y))


def panel_geometry(nx: int, ny: int, omega2: float, extent: float = 1.0) -> dict:
    """|T| (ny, nx), alpha of the x-faces (ny, nx + 1) and of the y-faces (ny + 1, nx) on the
    gnomonic panel [-extent, extent]^2 (extent 1: a full cube face) with nx x ny cells."""
    xs = -extent + 2.0 * extent * np.arange(nx + 1) / nx  # cell corners
    ys = -extent + 2.0 * extent * np.arange(ny + 1) / ny
    xc = -extent + 2.0 * extent * (np.arange(-1, nx + 1) + 0.5) / nx  # centres with the ghost ring
    yc = -extent + 2.0 * extent * (np.arange(-1, ny + 1) + 0.5) / ny
    F = _area_antiderivative(xs[None, :], ys[:, None])  # (ny + 1, nx + 1)
    area = F[1:, 1:] - F[1:, :-1] - F[:-1, 1:] + F[:-1, :-1]
    # x-face i (between cells i-1 and i) of row j: corners (xs[i], ys[j]), (xs[i], ys[j+1])
    e_x = arc(sphere_point(xs[None, :], ys[:-1, None]), sphere_point(xs[None, :], ys[1:, None]))
    d_x = arc(sphere_point(xc[None, :-1], yc[1:-1, None]), sphere_point(xc[None, 1:], yc[1:-1, None]))
    # y-face j (between rows j-1 and j) of column i
    e_y = arc(sphere_point(xs[None, :-1], ys[:, None]), sphere_point(xs[None, 1:], ys[:, None]))
    d_y = arc(sphere_point(xc[None, 1:-1], yc[:-1, None]), sphere_point(xc[None, 1:-1], yc[1:, None]))
    return {"area": np.ascontiguousarray(area), "ax": np.ascontiguousarray(-omega2 * e_x / d_x),
            "ay": np.ascontiguousarray(-omega2 * e_y / d_y)}


def radial_vectors(nz: int, H: float, omega2: float, lambda2: float):
    """a, b, c of Eq. (14) for nz cells on r in [1, 1 + H] (spacing h_z = H / nz)."""
    hz = H / nz
    rf = 1.0 + H * np.arange(nz + 1) / nz
    a = (rf[1:] ** 3 - rf[:-1] ** 3) / (3.0 * hz)
    b = -omega2 * lambda2 * rf[:-1] ** 2 / hz ** 2
    c = -omega2 * lambda2 * rf[1:] ** 2 / hz ** 2
    b[0] = 0.0
    c[-1] = 0.0
    return a, b, c


class PanelProblem:
    """Geometry of every multigrid level (1 = coarsest) and the radial vectors of one panel problem."""

    def __init__(self, nx, ny, nz, nlevels, omega2, lambda2, H, extent=1.0):
        self.nx, self.ny, self.nz, self.L = nx, ny, nz, nlevels
        self.levels = {}
        for l in range(nlevels, 0, -1):
            s = 2 ** (nlevels - l)
            self.levels[l] = panel_geometry(nx // s, ny // s, omega2, extent)
        self.a, self.b, self.c = radial_vectors(nz, H, omega2, lambda2)

    def geo(self, level=None):
        g = self.levels[self.L if level is None else level]
        return g["area"], g["ax"], g["ay"]

    def _args(self, level=None):
        area, ax, ay = self.geo(level)
        ny, nx = area.shape
        return [nx, ny, self.nz, _ptr(area), _ptr(ax), _ptr(ay), _ptr(self.a), _ptr(self.b), _ptr(self.c)]

    def apply_A(self, x, level=None):
        x = _f64(x)
        y = np.empty_like(x)
        _lib().orc_panel_apply_A(*self._args(level), _ptr(x), _ptr(y))
        return y

    def line_solve(self, r, level=None):
        r = _f64(r)
        x = np.empty_like(r)
        _lib().orc_panel_line_solve(*self._args(level), _ptr(r), _ptr(x))
        return x

    def residual(self, u, f, level=None):
        return _f64(f) - self.apply_A(u, level)

    def mg_solve(self, f, tol=1e-6, max_iter=100, u0=None, nu_pre=2, nu_post=2, n_coarse=2, rho=0.8):
        """V-cycles until ||r|| / ||r0|| < tol (Eq. (10)); returns (u, cycles, history, converged)."""
        f = _f64(f)
        u = np.zeros_like(f) if u0 is None else _f64(u0).copy()
        L = self.L
        nx = (ctypes.c_int * (L + 1))(*([0] + [self.levels[l]["area"].shape[1] for l in range(1, L + 1)]))
        ny = (ctypes.c_int * (L + 1))(*([0] + [self.levels[l]["area"].shape[0] for l in range(1, L + 1)]))
        ptrs = {}
        for key in ("area", "ax", "ay"):
            ptrs[key] = (ctypes.c_void_p * (L + 1))(*([None] + [self.levels[l][key].ctypes.data for l in range(1, L + 1)]))
        hist = np.zeros(max_iter + 1)
        conv = ctypes.c_int(0)
        it = _lib().orc_panel_mg_solve(L, ctypes.cast(nx, _P), ctypes.cast(ny, _P), self.nz,
                                       ctypes.cast(ptrs["area"], _P), ctypes.cast(ptrs["ax"], _P),
                                       ctypes.cast(ptrs["ay"], _P), _ptr(self.a), _ptr(self.b), _ptr(self.c),
                                       nu_pre, nu_post, n_coarse, rho, tol, max_iter, _ptr(f), _ptr(u), _ptr(hist),
                                       ctypes.byref(conv))
        if it < 0:
            raise ValueError("bad multigrid arguments")
        return u, it, hist[: it + 1], bool(conv.value)

    def cg_solve(self, f, tol=1e-6, max_iter=1000, u0=None):
        f = _f64(f)
        u = np.zeros_like(f) if u0 is None else _f64(u0).copy()
        hist = np.zeros(max_iter + 1)
        conv = ctypes.c_int(0)
        it = _lib().orc_panel_cg_solve(*self._args(), tol, max_iter, _ptr(f), _ptr(u), _ptr(hist), ctypes.byref(conv))
        return u, it, hist[: it + 1], bool(conv.value)


def restrict(rf):
    rf = _f64(rf)
    nz, nyf, nxf = rf.shape
    fc = np.empty((nz, nyf // 2, nxf // 2))
    _lib().orc_panel_restrict(nxf, nyf, nz, _ptr(rf), _ptr(fc))
    return fc


def prolongate_add(uc, uf):
    uc, uf = _f64(uc), _f64(uf).copy()
    nz, nyc, nxc = uc.shape
    _lib().orc_panel_prolongate_add(nxc, nyc, nz, _ptr(uc), _ptr(uf))
    return uf
