"""Test helpers that are independent of both the oracle's code and the CUDA path.

``spectral_solve`` is an exact solver for the constant-coefficient periodic/Neumann flat-box
operator built from library FFT/DCT routines and the closed-form eigenvalues; ``assemble`` turns
any matrix-free operator into a dense matrix by applying it to unit vectors.
"""
from __future__ import annotations

import math
import os

import numpy as np
import scipy.fft

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_golden(name: str) -> dict:
    """key value pairs from a tests/golden/*.txt fixture (comment lines start with #)."""
    out = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split(None, 1)
            out[key] = float(val)
    return out


def mode_eigs(nx, ny, nz):
    """sin^2 factors of the periodic (x, y) and Neumann (z) 1-D Laplacians, broadcastable."""
    sx = np.sin(np.pi * np.arange(nx) / nx) ** 2
    sy = np.sin(np.pi * np.arange(ny) / ny) ** 2
    sz = np.sin(np.pi * np.arange(nz) / (2 * nz)) ** 2
    return sx[None, None, :], sy[None, :, None], sz[:, None, None]


def mu_A(nx, ny, nz, cx, cy, v):
    sx, sy, sz = mode_eigs(nx, ny, nz)
    return 1.0 + 4 * cx * sx + 4 * cy * sy + 4 * v * sz


def mu_M(nx, ny, nz, cx, cy, v):
    _, _, sz = mode_eigs(nx, ny, nz)
    return 1.0 + 2 * cx + 2 * cy + 4 * v * sz + 0.0 * np.zeros((1, ny, nx))


def spectral_solve(f, cx, cy, v):
    """Exact A^{-1} f for constant v: Fourier in x and y, orthonormal DCT-II in z."""
    nz, ny, nx = f.shape
    fz = scipy.fft.dct(f, type=2, norm="ortho", axis=0)
    F = np.fft.fft2(fz, axes=(1, 2))
    U = F / mu_A(nx, ny, nz, cx, cy, v)
    uz = np.fft.ifft2(U, axes=(1, 2)).real
    return scipy.fft.idct(uz, type=2, norm="ortho", axis=0)


def fourier_dct_mode(nx, ny, nz, p, q, m, phase_x=0.0, phase_y=0.0):
    """cos(2 pi p i/nx + phase_x) cos(2 pi q j/ny + phase_y) cos(pi m (k+1/2)/nz)."""
    i = np.arange(nx)[None, None, :]
    j = np.arange(ny)[None, :, None]
    k = np.arange(nz)[:, None, None]
    return (np.cos(2 * np.pi * p * i / nx + phase_x) * np.cos(2 * np.pi * q * j / ny + phase_y)
            * np.cos(np.pi * m * (k + 0.5) / nz))


def assemble(apply, shape):
    """Dense matrix of a linear map on fields of the given input shape (column e = apply(unit e));
    the output may have another size (restriction, prolongation)."""
    n = int(np.prod(shape))
    cols = []
    for e in range(n):
        x = np.zeros(n)
        x[e] = 1.0
        cols.append(np.ravel(apply(x.reshape(shape))))
    return np.stack(cols, axis=1)


def cg_iteration_bound(kappa: float, tol: float) -> int:
    """Classical CG bound in the energy norm: ceil(sqrt(kappa)/2 * ln(2/tol))."""
    return int(math.ceil(0.5 * math.sqrt(kappa) * math.log(2.0 / tol)))


def rel(a, b) -> float:
    """||a - b||_2 / ||b||_2."""
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0))


def affine_network(cin, alpha, beta, gamma=0.0, nparams=None):
    """Flat parameters (W1 b1 W2 b2 W3 b3 W4 b4, W[co][ci][tap]) of the 4-layer network that computes
    NN(x) = alpha * x[0] + beta (+ gamma * relu(x[1]) when cin == 2) exactly: layer 1 splits channel 0
    into relu(x) and relu(-x) (centre taps +1 and -1) and copies relu(x[1]) to channel 2, layers 2
    and 3 pass channels 0..2 through (centre taps 1), layer 4 recombines them. All weights are
    powers of two or zero when alpha and gamma are, so BF16 holds them exactly."""
    n1, n2, n4 = 16 * cin * 27, 16 * 16 * 27, 16 * 27
    p = np.zeros(n1 + 16 + 2 * (n2 + 16) + n4 + 1 if nparams is None else nparams)
    W1 = p[:n1].reshape(16, cin, 27)
    W1[0, 0, 13], W1[1, 0, 13] = 1.0, -1.0
    if cin == 2:
        W1[2, 1, 13] = 1.0
    o2 = n1 + 16
    for o in (o2, o2 + n2 + 16):
        W = p[o:o + n2].reshape(16, 16, 27)
        W[0, 0, 13] = W[1, 1, 13] = W[2, 2, 13] = 1.0
    o4 = o2 + 2 * (n2 + 16)
    W4 = p[o4:o4 + n4].reshape(16, 27)
    W4[0, 13], W4[1, 13], W4[2, 13] = alpha, -alpha, gamma
    p[o4 + n4] = beta
    return p
