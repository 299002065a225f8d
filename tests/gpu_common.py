"""Shared fixtures of the GPU parity tests: build/load the CUDA library, move fields between numpy
and CUDA tensors, and the tolerances.

Tolerances (relative 2-norm error against the FP64 oracle):
  F64 and DW (double-word) kernels: 1e-10, the bound the method's FP64 applications must meet.
  F32 kernels: 2e-5. Derivation: the inputs are random, so no kernel output cancels by more than
  about a factor 10 relative to |A||x|; each output is a sum of at most 7 rounded products plus a
  Thomas sweep whose error grows at most linearly with nz (<= 128) on these diagonally dominant
  columns: 128 * 2^-24 * 10 ~ 8e-5 in the worst case, ~1e-6 observed; 2e-5 sits between.
"""
from __future__ import annotations

import numpy as np
import torch

from paper_1402_3545_gb300 import tpmg

TOL = {tpmg.F64: 1e-10, tpmg.DW: 1e-10, tpmg.F32: 2e-5}
UNIT_ROUNDOFF = {tpmg.F64: 2.0 ** -53, tpmg.DW: 2.0 ** -48, tpmg.F32: 2.0 ** -24}


def kappa_M(cx, cy, v) -> float:
    """Upper bound of the condition number of the column blocks M = D - v L_N (L_N the Neumann
    1-D Laplacian, spectrum in [0, 4)): 1 + 4 max(v) / (1 + 2cx + 2cy)."""
    return 1.0 + 4.0 * float(np.max(v)) / (1.0 + 2.0 * cx + 2.0 * cy)


def tol_inverse(prec: int, cx, cy, v) -> float:
    """Tolerance of kernels that apply M^{-1} (line solve, Smooth, RestrictSmooth, fused Tridiag):
    a backward-stable tridiagonal solve has forward error <= kappa(M) * (a few unit roundoffs);
    here 4 u kappa(M), never tighter than the plain tolerance of the precision. The double-word
    path runs levels with kappa(M) > 7000 (4 u kappa(M) > 1e-10) in native FP64, so 1e-10 holds there
    as well."""
    return max(TOL[prec], 4.0 * UNIT_ROUNDOFF[prec] * kappa_M(cx, cy, v)) if prec == tpmg.F32 else TOL[prec]
PRECS = [tpmg.F64, tpmg.DW, tpmg.F32]
PREC_IDS = ["f64", "dw", "f32"]


def dev(a: np.ndarray, prec: int) -> torch.Tensor:
    dt = torch.float32 if prec == tpmg.F32 else torch.float64
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dt)


def host(t: torch.Tensor) -> np.ndarray:
    torch.cuda.synchronize()
    return t.detach().double().cpu().numpy()


def rel(a, b) -> float:
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0))


def oracle_levels(cx: float, cy: float, v, L: int) -> dict:
    """The oracle's per-level coefficients: level L = finest (cx, cy, v); each coarser level has
    cx/4, cy/4 and v averaged over the 2x2 children (oracle.coarsen_v)."""
    import oracle
    out = {L: (cx, cy, np.asarray(v, dtype=np.float64))}
    for l in range(L - 1, 0, -1):
        c1, c2, vv = out[l + 1]
        out[l] = (c1 / 4.0, c2 / 4.0, oracle.coarsen_v(vv))
    return out


def make_problem(nx, ny, nz, omega2=1e-2, lam=None, seed=0):
    """A flat periodic box with hx = 1/nx, hy = 1/ny, hz = 1/nz and lambda^2 varying by column
    (the mid-size benchmark's field) unless a constant is given."""
    from paper_1402_3545_gb300 import workloads
    lam2 = workloads.lambda2_varying(nx, ny) if lam is None else lam
    return workloads.Problem(f"t{nx}x{ny}x{nz}", nx, ny, nz, omega2, 1.0 / nx, 1.0 / ny, 1.0 / nz, lam2,
                             workloads.levels_to_8(nx, ny), seed, "normal")
