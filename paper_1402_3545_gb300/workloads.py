"""Seeded synthetic workloads shaped like the paper's model problems.

This module only draws inputs: grid sizes, the PDE parameters omega^2, h, hz, the lambda^2 field
and right-hand sides. It holds none of the method's arithmetic (no stencil coefficients, no
operator, no solver); the CUDA library and the oracle each turn these parameters into their own
discrete coefficients. The paper measures only synthetic model problems (Sec. 5, "Problem- and
solver-parameters"), so seeded random fields stand in for data.

Fields are numpy float64 arrays of shape (nz, ny, nx), x fastest; lambda^2 is (ny, nx) or a
scalar.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Problem:
    """One elliptic problem -omega^2 (Lap_h u + lambda^2 d_zz u) + u = f on a flat periodic box."""

    name: str
    nx: int
    ny: int
    nz: int
    omega2: float
    hx: float
    hy: float
    hz: float
    lambda2: object  # float or (ny, nx) ndarray
    nlevels: int
    seed: int
    rhs_kind: str  # "uniform", "uniform_zero_mean" or "normal"

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def lambda2_field(self) -> np.ndarray:
        if np.ndim(self.lambda2) == 0:
            return np.full((self.ny, self.nx), float(self.lambda2))
        return np.asarray(self.lambda2, dtype=np.float64)

    def rhs(self) -> np.ndarray:
        return make_rhs(self.nx, self.ny, self.nz, self.seed, self.rhs_kind)


def make_rhs(nx: int, ny: int, nz: int, seed: int, kind: str) -> np.ndarray:
    """Seeded right-hand side in C order of (nz, ny, nx) from numpy's PCG64 generator."""
    rng = np.random.default_rng(seed)
    if kind == "normal":
        return rng.standard_normal((nz, ny, nx))
    f = rng.uniform(-1.0, 1.0, size=(nz, ny, nx))
    if kind == "uniform_zero_mean":
        f -= f.mean()
    elif kind != "uniform":
        raise ValueError(kind)
    return f


def levels_to_8(nx: int, ny: int) -> int:
    """Number of levels when halving both horizontal sizes while both are even and the larger one
    exceeds 8 (square grids: down to 8 x 8; elongated grids keep coarsening the long side, the short
    side may reach 1, so the coarsest level stays well conditioned)."""
    L = 1
    while nx % 2 == 0 and ny % 2 == 0 and max(nx, ny) > 8:
        nx //= 2
        ny //= 2
        L += 1
    return L


def lambda2_varying(nx: int, ny: int) -> np.ndarray:
    """lambda^2(x, y) = 1e3 (1 + 0.5 sin(2 pi x) cos(2 pi y)) at cell centres ((i+1/2)/nx, (j+1/2)/ny)."""
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    return 1e3 * (1.0 + 0.5 * np.sin(2 * np.pi * x)[None, :] * np.cos(2 * np.pi * y)[:, None])


def small(nx: int = 64, nz: int = 64) -> Problem:
    """Plain FP64 method, small: 64^2 x 64, h = hz = 1/64, omega^2 = 1e-2, lambda^2 = 1e3,
    uniform[-1,1] RHS from seed 0 with its mean removed, 4 levels."""
    return Problem("small_64x64x64", nx, nx, nz, 1e-2, 1.0 / nx, 1.0 / nx, 1.0 / nz, 1e3,
                   levels_to_8(nx, nx), 0, "uniform_zero_mean")


def mid(nx: int = 512, nz: int = 128) -> Problem:
    """FP64 mid-size: 512^2 x 128 with lambda^2(x, y) varying, N(0,1) RHS from seed 0, 7 levels."""
    return Problem(f"mid_{nx}x{nx}x{nz}_varlambda", nx, nx, nz, 1e-2, 1.0 / nx, 1.0 / nx,
                   1.0 / nz, lambda2_varying(nx, nx), levels_to_8(nx, nx), 0, "normal")


def mixed(nx: int = 1024, nz: int = 128) -> Problem:
    """Mixed precision: 1024^2 x 128, lambda^2 = 1e4, uniform[-1,1] RHS from seed 0, 8 levels."""
    return Problem(f"mixed_{nx}x{nx}x{nz}", nx, nx, nz, 1e-2, 1.0 / nx, 1.0 / nx, 1.0 / nz, 1e4,
                   levels_to_8(nx, nx), 0, "uniform")


def learned_target(nx: int = 2048, nz: int = 64) -> Problem:
    """Learned-preconditioner application grid: 2048^2 x 64, lambda^2 = 1e3, h = 1/2048."""
    return Problem(f"learned_{nx}x{nx}x{nz}", nx, nx, nz, 1e-2, 1.0 / nx, 1.0 / nx, 1.0 / nz,
                   1e3, levels_to_8(nx, nx), 0, "uniform")


def paper_shaped(nx: int = 512, nz: int = 128, lambda2: float = 1e3, nu_cfl: float = 8.4,
                 nlevels: int | None = None) -> Problem:
    """Paper-shaped variant: omega = nu_CFL h / 2 with the horizontal CFL number nu_CFL = 2 omega / h
    of Sec. 5.2 (8.4 by default, i.e. omega = 4.2 h, Eq. (4)), so kappa ~ 1 + 2 nu_CFL^2 (Eq. (7):
    142 at 8.4); N(0,1) right-hand side from seed 0."""
    h = 1.0 / nx
    name = f"paper_shaped_{nx}x{nx}x{nz}" + ("" if nu_cfl == 8.4 else f"_cfl{nu_cfl:g}")
    return Problem(name, nx, nx, nz, (0.5 * nu_cfl * h) ** 2, h, h, 1.0 / nz,
                   lambda2, levels_to_8(nx, nx) if nlevels is None else nlevels, 0, "normal")


# The robustness study of Sec. 5.2 (512^2 x 128 in the paper): nu_CFL from 0.84 to 840 with 5, 7 and
# 10 multigrid levels; the number of smoothing steps on the coarsest level grows with nu_CFL as the
# paper reports it needed (10 levels: 2 throughout; 7 levels: 5 at 84, 15 at 840; 5 levels: 30 at
# 84, 150 at 840; 2 up to 16.8).
ROBUSTNESS_CFL = (0.84, 8.4, 84.0, 840.0)
ROBUSTNESS_LEVELS = (5, 7, 10)


def robustness_coarse_steps(nlevels: int, nu_cfl: float) -> int:
    """Smoothing steps on the coarsest level for the robustness study (Sec. 5.2)."""
    if nu_cfl <= 16.8 or nlevels >= 10:
        return 2
    table = {7: {84.0: 5, 840.0: 15}, 5: {84.0: 30, 840.0: 150}}
    row = table.get(nlevels, table[5] if nlevels < 7 else table[7])
    return row[min(row, key=lambda c: abs(c - nu_cfl))]


@dataclasses.dataclass
class PanelProblem:
    """The paper's own problem, Eq. (1) on one gnomonic cubed-sphere panel (Sec. 2.1.1): nx x ny
    cells on the panel, nz on r in [1, 1 + H], omega^2, lambda^2, the panel's half-width in cube-face
    coordinates (1: a whole cube face)."""

    name: str
    nx: int
    ny: int
    nz: int
    omega2: float
    lambda2: float
    H: float
    extent: float
    nlevels: int
    seed: int
    rhs_kind: str

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz

    def rhs(self) -> np.ndarray:
        return make_rhs(self.nx, self.ny, self.nz, self.seed, self.rhs_kind)


def panel(nx: int = 512, nz: int = 128, nu_cfl: float = 8.4, nlevels: int = 5) -> PanelProblem:
    """The paper's single-GPU configuration on its own operator: an nx x nx panel (mean angular cell
    width h = (pi/2) / nx), omega = nu_CFL h / 2 (Eq. (4), nu_CFL = 8.4), lambda^2 = 1 (the limit of
    lambda(h) at high resolution, Sec. 2.1; the table of the companion paper is not available), an
    atmosphere 10 km deep on the earth's 6371 km radius (H = 10/6371), 5 levels, N(0,1) right-hand
    side from seed 0."""
    h = 0.5 * np.pi / nx
    return PanelProblem(f"panel_{nx}x{nx}x{nz}", nx, nx, nz, (0.5 * nu_cfl * h) ** 2, 1.0, 10.0 / 6371.0, 1.0,
                        nlevels, 0, "normal")


def batched(nprob: int = 64, seed: int = 0) -> list[Problem]:
    """Batched: sizes drawn uniformly from {64,128,256,512}^2 x {32,64,128} (seed 0), lambda^2
    log-uniform in [1e2, 1e4], problem b's uniform[-1,1] RHS from seed 1000 + b. Horizontal cells are
    square, hx = hy = 1/max(nx, ny) (the unit square spans the longer side), hz = 1/nz."""
    rng = np.random.default_rng(seed)
    probs = []
    for b in range(nprob):
        nx = int(rng.choice([64, 128, 256, 512]))
        ny = int(rng.choice([64, 128, 256, 512]))
        nz = int(rng.choice([32, 64, 128]))
        lam2 = float(10.0 ** rng.uniform(2.0, 4.0))
        h = 1.0 / max(nx, ny)
        probs.append(Problem(f"batch{b}", nx, ny, nz, 1e-2, h, h, 1.0 / nz, lam2,
                             levels_to_8(nx, ny), 1000 + b, "uniform"))
    return probs


def scaled_down(p: Problem, nx: int, ny: int | None = None, nz: int | None = None) -> Problem:
    """The same problem family at a smaller size (for parity tests the oracle finishes quickly)."""
    ny = nx if ny is None else ny
    nz = p.nz if nz is None else nz
    lam = p.lambda2
    if np.ndim(lam) != 0:
        lam = lambda2_varying(nx, ny)
    return Problem(p.name + f"_scaled_{nx}x{ny}x{nz}", nx, ny, nz, p.omega2, 1.0 / nx, 1.0 / ny,
                   1.0 / nz, lam, levels_to_8(nx, ny), p.seed, p.rhs_kind)

