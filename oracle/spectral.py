"""Exact solve of the constant-coefficient flat-box problem (test infrastructure, part of the oracle).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py`` may import this
module; the CUDA library never calls it.

With a constant vertical coefficient v the operator of Sec. 2.1.1 (periodic in x and y, Neumann with
the mirror ghost cell at the bottom and top) is diagonal in the basis of discrete Fourier modes in x
and y times DCT-II modes cos(pi m (k + 1/2) / nz) in z, with eigenvalue

    mu(p, q, m) = 1 + 4 cx sin^2(pi p / nx) + 4 cy sin^2(pi q / ny) + 4 v sin^2(pi m / (2 nz))

(the closed form behind the condition-number estimate of Eq. (7)). So A^{-1} f is the transform of
f divided by mu and transformed back: the exact solution up to the rounding of the transforms, the
reference against which full-size solutions of such problems are measured. Library FFT and DCT
routines do the transforms; nothing here shares code with the multigrid oracle or the CUDA path.
"""
from __future__ import annotations

import numpy as np
import scipy.fft


def eigenvalues_plane(nx: int, ny: int, nz: int, cx: float, cy: float, v: float, m: int) -> np.ndarray:
    """mu(p, q, m) for one vertical mode m on the half spectrum p = 0..nx//2 of a real transform in
    x (sin^2(pi p / nx) is the same for p and nx - p), shape (ny, nx//2 + 1)."""
    sx = np.sin(np.pi * np.arange(nx // 2 + 1) / nx) ** 2
    sy = np.sin(np.pi * np.arange(ny) / ny) ** 2
    sz = np.sin(np.pi * m / (2 * nz)) ** 2
    return 1.0 + 4.0 * cx * sx[None, :] + 4.0 * cy * sy[:, None] + 4.0 * v * sz


def exact_solve(f: np.ndarray, cx: float, cy: float, v, workers: int = -1) -> np.ndarray:
    """u = A^{-1} f for a constant v (a number, or a field of equal values); f has shape
    (nz, ny, nx), x fastest. `workers` host threads
    run the transforms (-1: all cores). Peak memory is about three copies of f."""
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = f.shape
    va = np.asarray(v, dtype=np.float64)
    if va.size > 1 and not np.all(va == va.ravel()[0]):
        raise ValueError("exact_solve needs a constant vertical coefficient")
    v = float(va.ravel()[0])
    g = scipy.fft.dct(f, type=2, norm="ortho", axis=0, workers=workers)  # vertical modes m
    for m in range(nz):  # one plane at a time keeps the complex spectrum to one plane
        F = scipy.fft.rfft2(g[m], workers=workers)
        F /= eigenvalues_plane(nx, ny, nz, cx, cy, v, m)
        g[m] = scipy.fft.irfft2(F, s=(ny, nx), workers=workers)
    return scipy.fft.idct(g, type=2, norm="ortho", axis=0, workers=workers, overwrite_x=True)
