"""Oracle: plain, slow FP64 CPU implementation of the method (test infrastructure only).

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this package. The CUDA library shares no code with it. Fields are numpy float64 arrays of
shape (nz, ny, nx) (x fastest); the vertical coefficient ``v`` is an (ny, nx) array of
omega^2 lambda^2 / hz^2 per column. Each wrapper names the passage of the paper it follows; the C
source (``tpmg_oracle.c``) holds the arithmetic, with OpenMP over cells and columns where the host
compiler has it (``set_threads``; results do not depend on the thread count). ``oracle.spectral``
is the exact solver of constant-coefficient problems (library FFT/DCT and the closed-form
eigenvalues), the reference for full-size solutions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tpmg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_D = ctypes.c_double
_I = ctypes.c_int
_P = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/liboracle.so with the host gcc (no -march flags)."""
    srcs = [_SRC] + [os.path.join(_HERE, s) for s in ("nn_oracle.c", "panel_oracle.c")
                     if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs)
    import platform
    stamp = _LIB + ".host"
    if not os.path.exists(stamp) or open(stamp).read() != platform.machine():
        force = True  # built on another host architecture
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        # OpenMP over cells and columns where the host compiler has it (results do not depend on
        # the thread count: see orc_set_threads), else the same code on one thread
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", _LIB] + srcs + ["-lm"]
        if subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True).returncode != 0:
            subprocess.run(base, check=True)
        with open(stamp, "w") as fh:
            fh.write(platform.machine())
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        for name, args, res in [
            ("orc_set_threads", [_I], _I),
            ("orc_apply_A", [_I, _I, _I, _D, _D, _P, _P, _P], None),
            ("orc_line_solve", [_I, _I, _I, _D, _D, _P, _P, _P], None),
            ("orc_residual", [_I, _I, _I, _D, _D, _P, _P, _P, _P], None),
            ("orc_smooth", [_I, _I, _I, _D, _D, _P, _D, _P, _P, _P], None),
            ("orc_restrict", [_I, _I, _I, _P, _P], None),
            ("orc_prolongate_add", [_I, _I, _I, _P, _P], None),
            ("orc_coarsen_v", [_I, _I, _P, _P], None),
            ("orc_vcycle", [_I, _I, _I, _I, _D, _D, _P, _I, _I, _I, _D, _P, _P], _I),
            ("orc_mg_solve", [_I, _I, _I, _I, _D, _D, _P, _I, _I, _I, _D, _D, _I, _P, _P, _P, _P], _I),
            ("orc_cg_solve", [_I, _I, _I, _D, _D, _P, _D, _I, _P, _P, _P, _P], _I),
            ("orc_ir_solve", [_I, _I, _I, _I, _D, _D, _P, _I, _I, _I, _D, _D, _I, _P, _P, _P, _P], _I),
        ]:
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def set_threads(n: int = 0) -> int:
    """Host threads of the oracle's loops over cells and columns (n >= 1; 0 leaves the count as it
    is); returns the count in effect. Results are the same for every count: each cell or column is
    computed by the same code, and dot products and norms run in index order on one thread."""
    return int(_load().orc_set_threads(int(n)))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _vcol(v, nx, ny) -> np.ndarray:
    v = np.asarray(v, dtype=np.float64)
    if v.ndim == 0:
        v = np.full((ny, nx), float(v))
    assert v.shape == (ny, nx), v.shape
    return np.ascontiguousarray(v)


def coefficients(omega2, hx, hy, hz, lambda2):
    """Discrete coefficients of the flat-box operator (Sec. 2.1.1): cx = omega^2/hx^2,
    cy = omega^2/hy^2 and v = omega^2 lambda^2/hz^2 (per column when lambda^2 is a field)."""
    return omega2 / hx ** 2, omega2 / hy ** 2, omega2 * np.asarray(lambda2, dtype=np.float64) / hz ** 2


def problem_coefficients(p):
    """coefficients() for a workloads.Problem."""
    return coefficients(p.omega2, p.hx, p.hy, p.hz, p.lambda2_field())


def apply_A(x, cx, cy, v):
    """y = A x, Sec. 2.1.1 (flat-box entries of Eq. (6)) with periodic x/y and Neumann z ends."""
    x = _f64(x)
    nz, ny, nx = x.shape
    v = _vcol(v, nx, ny)
    y = np.empty_like(x)
    _load().orc_apply_A(nx, ny, nz, cx, cy, _ptr(v), _ptr(x), _ptr(y))
    return y


def line_solve(b, cx, cy, v):
    """x = M^{-1} b, vertical line relaxation by the Thomas algorithm (Sec. 2.2)."""
    b = _f64(b)
    nz, ny, nx = b.shape
    v = _vcol(v, nx, ny)
    x = np.empty_like(b)
    _load().orc_line_solve(nx, ny, nz, cx, cy, _ptr(v), _ptr(b), _ptr(x))
    return x


def residual(u, f, cx, cy, v):
    """r = f - A u (Residual kernel, Sec. 3.1)."""
    u, f = _f64(u), _f64(f)
    nz, ny, nx = u.shape
    v = _vcol(v, nx, ny)
    r = np.empty_like(u)
    _load().orc_residual(nx, ny, nz, cx, cy, _ptr(v), _ptr(u), _ptr(f), _ptr(r))
    return r


def smooth(u, f, cx, cy, v, rho):
    """u + rho M^{-1}(f - A u), Eq. (11) "MultigridSmoother"."""
    u, f = _f64(u), _f64(f)
    nz, ny, nx = u.shape
    v = _vcol(v, nx, ny)
    out = np.empty_like(u)
    _load().orc_smooth(nx, ny, nz, cx, cy, _ptr(v), rho, _ptr(u), _ptr(f), _ptr(out))
    return out


def restrict(rf):
    """Cell-average restriction, horizontal only (Sec. 2.2)."""
    rf = _f64(rf)
    nz, nyf, nxf = rf.shape
    fc = np.empty((nz, nyf // 2, nxf // 2))
    _load().orc_restrict(nxf, nyf, nz, _ptr(rf), _ptr(fc))
    return fc


def prolongate_add(uc, uf):
    """uf + P uc, horizontal bilinear interpolation of cell-centred data (Sec. 2.2)."""
    uc = _f64(uc)
    out = _f64(uf).copy()
    nz, nyc, nxc = uc.shape
    assert out.shape == (nz, 2 * nyc, 2 * nxc)
    _load().orc_prolongate_add(nxc, nyc, nz, _ptr(uc), _ptr(out))
    return out


def coarsen_v(vf):
    """Coarse-level vertical coefficient: average of the 2x2 children."""
    vf = _f64(vf)
    nyf, nxf = vf.shape
    vc = np.empty((nyf // 2, nxf // 2))
    _load().orc_coarsen_v(nxf, nyf, _ptr(vf), _ptr(vc))
    return vc


def vcycle(u, f, cx, cy, v, nlevels, nu_pre=2, nu_post=2, n_coarse=2, rho=0.8):
    """One V-cycle of Algorithm 1 (generalised to nu_pre/nu_post smoothing steps)."""
    u = _f64(u).copy()
    f = _f64(f)
    nz, ny, nx = u.shape
    v = _vcol(v, nx, ny)
    rc = _load().orc_vcycle(nx, ny, nz, nlevels, cx, cy, _ptr(v), nu_pre, nu_post, n_coarse,
                            rho, _ptr(f), _ptr(u))
    if rc != 0:
        raise ValueError("bad multigrid arguments")
    return u


def mg_solve(f, cx, cy, v, nlevels, tol=1e-6, max_iter=100, u0=None, nu_pre=2, nu_post=2,
             n_coarse=2, rho=0.8):
    """V-cycles until ||r||/||r0|| < tol, Eq. (10). Returns (u, iters, history, converged)."""
    f = _f64(f)
    nz, ny, nx = f.shape
    v = _vcol(v, nx, ny)
    u = np.zeros_like(f) if u0 is None else _f64(u0).copy()
    hist = np.zeros(max_iter + 1)
    conv = ctypes.c_int(0)
    it = _load().orc_mg_solve(nx, ny, nz, nlevels, cx, cy, _ptr(v), nu_pre, nu_post, n_coarse,
                              rho, tol, max_iter, _ptr(f), _ptr(u), _ptr(hist),
                              ctypes.byref(conv))
    if it < 0:
        raise ValueError("bad multigrid arguments")
    return u, it, hist[: it + 1], bool(conv.value)


def cg_solve(f, cx, cy, v, tol=1e-6, max_iter=1000, u0=None):
    """Line-preconditioned CG (Sec. 2.2). Returns (u, iters, history, converged)."""
    f = _f64(f)
    nz, ny, nx = f.shape
    v = _vcol(v, nx, ny)
    u = np.zeros_like(f) if u0 is None else _f64(u0).copy()
    hist = np.zeros(max_iter + 1)
    conv = ctypes.c_int(0)
    it = _load().orc_cg_solve(nx, ny, nz, cx, cy, _ptr(v), tol, max_iter, _ptr(f), _ptr(u),
                              _ptr(hist), ctypes.byref(conv))
    return u, it, hist[: it + 1], bool(conv.value)


def ir_solve(f, cx, cy, v, nlevels, tol=1e-6, max_iter=100, u0=None, nu_pre=2, nu_post=2,
             n_coarse=2, rho=0.8):
    """Iterative refinement with one V-cycle per correction. Returns (u, iters, hist, conv)."""
    f = _f64(f)
    nz, ny, nx = f.shape
    v = _vcol(v, nx, ny)
    u = np.zeros_like(f) if u0 is None else _f64(u0).copy()
    hist = np.zeros(max_iter + 1)
    conv = ctypes.c_int(0)
    it = _load().orc_ir_solve(nx, ny, nz, nlevels, cx, cy, _ptr(v), nu_pre, nu_post, n_coarse,
                              rho, tol, max_iter, _ptr(f), _ptr(u), _ptr(hist),
                              ctypes.byref(conv))
    if it < 0:
        raise ValueError("bad multigrid arguments")
    return u, it, hist[: it + 1], bool(conv.value)


# ------------------------------------------------------------------ learned stage and flexible CG
class _OrcPrec(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("L", ctypes.c_int), ("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int),
                ("n_coarse", ctypes.c_int), ("rho", ctypes.c_double), ("cin", ctypes.c_int),
                ("params", ctypes.c_void_p), ("aux", ctypes.c_void_p), ("nn_used", ctypes.c_int),
                ("nn_rejected", ctypes.c_int)]


def _nnlib():
    lib = _load()
    if not getattr(lib, "_nn_ready", False):
        for name, args, res in [
            ("orc_conv3d_fwd", [_I, _I, _I, _I, _I, _P, _P, _I, _P, _P], None),
            ("orc_conv3d_bwd", [_I, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P], None),
            ("orc_nn_forward", [_I, _I, _I, _I, _P, _P, _P, _P], None),
            ("orc_nn_loss_grad", [_I, _I, _I, _I, _P, _P, _P, _P], _D),
            ("orc_nn_loss_grad_residual", [_I, _I, _I, _I, _D, _D, _P, _P, _P, _P], _D),
            ("orc_diag_inv", [_I, _I, _I, _D, _D, _P, _P], None),
            ("orc_fcg_precondition", [_I, _I, _I, _D, _D, _P, ctypes.POINTER(_OrcPrec), _P, _P, _P], None),
            ("orc_adam_step", [ctypes.c_size_t, _P, _P, _P, _P, _I, _D, _D, _D, _D], None),
            ("orc_fcg_solve", [_I, _I, _I, _D, _D, _P, ctypes.POINTER(_OrcPrec), _D, _I, _P, _P, _P, _P], _I),
            ("orc_nn_nparams", [_I], ctypes.c_size_t),
        ]:
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        lib._nn_ready = True
    return lib


def nn_nparams(cin: int) -> int:
    return int(_nnlib().orc_nn_nparams(cin))


def conv3d(x, W, b, relu=False):
    """Cross-correlation with 3x3x3 kernels, circular in x and y, zero-padded in z.
    x: (cin, nz, ny, nx); W: (cout, cin, 3, 3, 3); b: (cout,) or None."""
    x = _f64(x)
    W = _f64(W)
    cin, nz, ny, nx = x.shape
    cout = W.shape[0]
    y = np.empty((cout, nz, ny, nx))
    bb = None if b is None else _f64(b)
    _nnlib().orc_conv3d_fwd(nx, ny, nz, cin, cout, _ptr(W), None if bb is None else _ptr(bb), int(relu),
                            _ptr(x), _ptr(y))
    return y


def conv3d_backward(x, W, dy, want_dx=True):
    """(dx, dW, db) of one layer for the gradient dy of its output."""
    x, W, dy = _f64(x), _f64(W), _f64(dy)
    cin, nz, ny, nx = x.shape
    cout = W.shape[0]
    dx = np.empty_like(x) if want_dx else None
    dW = np.zeros_like(W)
    db = np.zeros(cout)
    _nnlib().orc_conv3d_bwd(nx, ny, nz, cin, cout, _ptr(W), _ptr(x), _ptr(dy), None if dx is None else _ptr(dx),
                            _ptr(dW), _ptr(db))
    return dx, dW, db


def nn_forward(params, x):
    """The 4-layer network (cin -> 16 -> 16 -> 16 -> 1); x: (cin, nz, ny, nx); returns (nz, ny, nx)."""
    params, x = _f64(params), _f64(x)
    cin, nz, ny, nx = x.shape
    out = np.empty((nz, ny, nx))
    _nnlib().orc_nn_forward(nx, ny, nz, cin, _ptr(params), _ptr(x), _ptr(out), None)
    return out


def nn_loss_grad(params, x, target):
    """Mean-squared loss of the network output against target, and its parameter gradient."""
    params, x, target = _f64(params), _f64(x), _f64(target)
    cin, nz, ny, nx = x.shape
    g = np.empty_like(params)
    loss = _nnlib().orc_nn_loss_grad(nx, ny, nz, cin, _ptr(params), _ptr(x), _ptr(target), _ptr(g))
    return loss, g


def diag_inv(shape, cx, cy, v):
    """1 / diag(A) per cell, shape (nz, ny, nx): the unit of the network's output."""
    nz, ny, nx = shape
    v = _vcol(v, nx, ny)
    out = np.empty(shape)
    _nnlib().orc_diag_inv(nx, ny, nz, cx, cy, _ptr(v), _ptr(out))
    return out


def nn_loss_grad_residual(params, x, cx, cy, v):
    """Residual loss mean((x[0] - A D^-1 NN(x))^2), D = diag(A), for the operator (cx, cy, v) and
    its parameter gradient."""
    params, x = _f64(params), _f64(x)
    cin, nz, ny, nx = x.shape
    v = _vcol(v, nx, ny)
    g = np.empty_like(params)
    loss = _nnlib().orc_nn_loss_grad_residual(nx, ny, nz, cin, cx, cy, _ptr(v), _ptr(params), _ptr(x), _ptr(g))
    return loss, g


def adam_step(theta, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on theta, m, v (float64 numpy arrays)."""
    g = _f64(g)
    _nnlib().orc_adam_step(theta.size, _ptr(theta), _ptr(g), _ptr(m), _ptr(v), t, lr, beta1, beta2, eps)


def fcg_precondition(r, cx, cy, v, mode=1, nlevels=1, params=None, aux=None, nu_pre=2, nu_post=2, n_coarse=2,
                     rho=0.8):
    """One application of flexible CG's preconditioner to r: (z, learned candidate, kept)."""
    r = _f64(r)
    nz, ny, nx = r.shape
    v = _vcol(v, nx, ny)
    z = np.zeros_like(r)
    cand = np.full_like(r, np.nan)
    pp = None if params is None else _f64(params)
    ax = None if aux is None else _f64(np.broadcast_to(np.asarray(aux, dtype=np.float64), (nz, ny, nx)))
    P = _OrcPrec(mode, nlevels, nu_pre, nu_post, n_coarse, rho, 1 if ax is None else 2,
                 None if pp is None else pp.ctypes.data, None if ax is None else ax.ctypes.data, 0, 0)
    _nnlib().orc_fcg_precondition(nx, ny, nz, cx, cy, _ptr(v), ctypes.byref(P), _ptr(r), _ptr(z), _ptr(cand))
    return z, cand, bool(P.nn_used)


def fcg_solve(f, cx, cy, v, mode=1, nlevels=1, tol=1e-6, max_iter=500, params=None, aux=None, u0=None,
              nu_pre=2, nu_post=2, n_coarse=2, rho=0.8):
    """Flexible CG(1); mode 0: line-solve preconditioner, 1: V-cycle, 2: V-cycle + learned stage.
    aux: the network's second input channel, per column (ny, nx) or per cell (nz, ny, nx).
    Returns (u, iters, history, converged, nn_used, nn_rejected)."""
    f = _f64(f)
    nz, ny, nx = f.shape
    v = _vcol(v, nx, ny)
    u = np.zeros_like(f) if u0 is None else _f64(u0).copy()
    hist = np.zeros(max_iter + 1)
    conv = ctypes.c_int(0)
    pp = None if params is None else _f64(params)
    ax = None if aux is None else _f64(np.broadcast_to(np.asarray(aux, dtype=np.float64), (nz, ny, nx)))
    P = _OrcPrec(mode, nlevels, nu_pre, nu_post, n_coarse, rho, 1 if ax is None else 2,
                 None if pp is None else pp.ctypes.data, None if ax is None else ax.ctypes.data, 0, 0)
    it = _nnlib().orc_fcg_solve(nx, ny, nz, cx, cy, _ptr(v), ctypes.byref(P), tol, max_iter, _ptr(f), _ptr(u),
                                _ptr(hist), ctypes.byref(conv))
    return u, it, hist[: it + 1], bool(conv.value), P.nn_used, P.nn_rejected
