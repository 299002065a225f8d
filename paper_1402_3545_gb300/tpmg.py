"""Thin ctypes binding of the C ABI in include/tpmg.h (libtpmg.so, built in-tree).

Each function here has the name of the C entry point without its ``tpmg_`` prefix and only
marshals arguments: torch CUDA tensors become device pointers, the current torch stream becomes
the cudaStream_t, and a non-OK status becomes a ``TpmgError``. Every computation runs in the CUDA
library; there is no CPU fallback -- importing this module without the built library raises.

Fields are contiguous CUDA tensors of shape (nz, ny, nx): float64 for F64, DW and MIXED, float32
for F32. Levels are numbered 1 (coarsest) .. L (finest) as in the paper's Sec. 2.2.
"""
from __future__ import annotations

import ctypes
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtpmg.so")

F64, F32, DW, MIXED = 0, 1, 2, 3
PREC = {"f64": F64, "f32": F32, "dw": DW, "mixed": MIXED}
STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
          4: "not converged", 5: "non-finite value", 6: "device wait timed out",
          7: "learned stage rejected"}
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_NOT_CONVERGED, ERR_NONFINITE, ERR_TIMEOUT, ERR_NN_REJECTED = range(8)


class TpmgError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({msg})")
        self.status = status


class Params(ctypes.Structure):
    _fields_ = [("nu_pre", ctypes.c_int), ("nu_post", ctypes.c_int), ("n_coarse", ctypes.c_int),
                ("max_iter", ctypes.c_int), ("rho", ctypes.c_double), ("tol", ctypes.c_double),
                ("prec", ctypes.c_int), ("use_graph", ctypes.c_int), ("timeout_s", ctypes.c_double),
                ("zero_guess", ctypes.c_int), ("coarse_bf16", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("rel_res", ctypes.c_double),
                ("r0", ctypes.c_double), ("history", ctypes.POINTER(ctypes.c_double)),
                ("history_len", ctypes.c_int), ("ms", ctypes.c_double)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
# tpmg_alloc_fn / tpmg_free_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_SIGNATURES = {
    "tpmg_create_grid": [_I, _I, _I, _I, ctypes.POINTER(_P)],
    "tpmg_destroy_grid": [_P],
    "tpmg_grid_nlevels": [_P],
    "tpmg_grid_level_size": [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)],
    "tpmg_create_operator": [_P, _D, _D, _D, _D, _D, _P, ctypes.POINTER(_P)],
    "tpmg_destroy_operator": [_P],
    "tpmg_op_reserve": [_P, _I],
    "tpmg_op_level_coefficients": [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), _P],
    "tpmg_apply_A": [_P, _I, _I, _P, _P, _P],
    "tpmg_line_solve": [_P, _I, _I, _P, _P, _P],
    "tpmg_smooth": [_P, _I, _I, _D, _P, _P, _P, _P, _P],
    "tpmg_residual": [_P, _I, _I, _P, _P, _P, _P, _P],
    "tpmg_restrict_smooth": [_P, _I, _I, _D, _P, _P, _P, _P],
    "tpmg_residual_restrict_smooth": [_P, _I, _I, _D, _P, _P, _P, _P, _P],
    "tpmg_set_fusion": [_P, _I],
    "tpmg_set_allocator": [ALLOC_FN, FREE_FN, _P],
    "tpmg_prolongate": [_P, _I, _I, _P, _P, _P],
    "tpmg_cg_fused_spmv": [_P, _I, _D, _D, _P, _P, _P, _P, _P, _P],
    "tpmg_cg_fused_tridiag": [_P, _I, _D, _P, _P, _P, _P, _P, _P],
    "tpmg_default_params": [ctypes.POINTER(Params)],
    "tpmg_mg_solve": [_P, ctypes.POINTER(Params), _P, _P, ctypes.POINTER(Info), _P],
    "tpmg_mg_solve_host": [_P, ctypes.POINTER(Params), _I, _P, _P, ctypes.POINTER(Info), _P, _P],
    "tpmg_create_panel_operator": [_P, _D, _D, _D, _D, ctypes.POINTER(_P)],
    "tpmg_panel_level_geometry": [_P, _I, _P, _P, _P],
    "tpmg_panel_apply_A": [_P, _I, _P, _P, _P],
    "tpmg_panel_line_solve": [_P, _I, _P, _P, _P],
    "tpmg_panel_smooth": [_P, _I, _D, _P, _P, _P, _P, _P],
    "tpmg_panel_residual": [_P, _I, _P, _P, _P, _P, _P],
    "tpmg_panel_restrict_smooth": [_P, _I, _D, _P, _P, _P, _P],
    "tpmg_panel_prolongate": [_P, _I, _P, _P, _P],
    "tpmg_vcycle": [_P, ctypes.POINTER(Params), _P, _P, _P],
    "tpmg_cg_solve": [_P, ctypes.POINTER(Params), _P, _P, ctypes.POINTER(Info), _P],
    "tpmg_mg_solve_batched": [_I, _P, ctypes.POINTER(Params), _P, _P, _P, _P],
    "tpmg_nn_nparams": [_I],
    "tpmg_nn_create": [_I, _P, ctypes.POINTER(_P)],
    "tpmg_nn_destroy": [_P],
    "tpmg_nn_get_params": [_P, _P],
    "tpmg_nn_set_params": [_P, _P],
    "tpmg_nn_forward": [_P, _I, _I, _I, _P, _P, _P],
    "tpmg_nn_loss_grad": [_P, _I, _I, _I, _P, _P, _P, _P, _P],
    "tpmg_nn_train_step": [_P, _I, _I, _I, _P, _P, _D, _P, _P],
    "tpmg_nn_loss_grad_residual": [_P, _P, _P, _P, _P, _P],
    "tpmg_nn_train_step_residual": [_P, _P, _P, _D, _P, _P],
    "tpmg_nn_make_pair": [_P, _I, _P, _P, _P, _P, _P, _P, _P],
    "tpmg_fcg_solve": [_P, _P, _P, ctypes.POINTER(Params), _P, _P, ctypes.POINTER(Info), ctypes.POINTER(_I), _P],
    "tpmg_residual_norm_noalloc": [_I, _I, _I, _D, _D, _P, _P, _P, _P, _P, _P],
    "tpmg_noalloc_last_error": [],
    "tpmg_time_kernel": [_P, _I, _I, _I, ctypes.POINTER(_D), _P],
    "tpmg_kernel_launches": [],
    "tpmg_measure_alu_rate": [_I, _I, _P, _P],
    "tpmg_autotune": [_P, _I, _I, _P, _P],
    "tpmg_set_variant": [_P, _I, _I, _I],
    "tpmg_status_string": [_I],
    "tpmg_last_error": [],
}

(K_SMOOTH, K_RESIDUAL, K_APPLY_A, K_LINE_SOLVE, K_RESTRICT_SMOOTH, K_PROLONGATE, K_CG_SPMV, K_CG_TRIDIAG,
 K_RESIDUAL_RESTRICT) = range(9)


def load():
    """Loads libtpmg.so (raises if it has not been built: there is no fallback path)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (nvcc, sm_103a)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = _I
        lib.tpmg_status_string.restype = ctypes.c_char_p
        lib.tpmg_last_error.restype = ctypes.c_char_p
        lib.tpmg_noalloc_last_error.restype = ctypes.c_char_p
        lib.tpmg_grid_nlevels.restype = _I
        lib.tpmg_default_params.restype = None
        lib.tpmg_kernel_launches.restype = ctypes.c_ulonglong
        _lib = lib
    return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def _check(status: int, where: str, allow=()):
    if status != OK and status not in allow:
        raise TpmgError(status, where, load().tpmg_last_error().decode())
    return status


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _dtype(prec: int):
    return torch.float32 if prec == F32 else torch.float64


def _field(t: torch.Tensor, prec: int, numel: int, name: str) -> int:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != _dtype(prec):
        raise TypeError(f"{name} must be {_dtype(prec)} for precision {prec}, got {t.dtype}")
    if not t.is_contiguous() or t.numel() != numel:
        raise ValueError(f"{name} must be contiguous with {numel} elements")
    return t.data_ptr()


def _scalar_out(t) -> int | None:
    if t is None:
        return None
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.numel() >= 1):
        raise TypeError("scalar outputs are CUDA float64 tensors")
    return t.data_ptr()


# ---------------------------------------------------------------- grid and operator
def create_grid(nx: int, ny: int, nz: int, nlevels: int = 0) -> int:
    h = _P()
    _check(load().tpmg_create_grid(nx, ny, nz, nlevels, ctypes.byref(h)), "create_grid")
    return h.value


def destroy_grid(g: int) -> None:
    load().tpmg_destroy_grid(g)


def grid_nlevels(g: int) -> int:
    return load().tpmg_grid_nlevels(g)


def grid_level_size(g: int, level: int) -> tuple[int, int]:
    nx, ny = _I(), _I()
    _check(load().tpmg_grid_level_size(g, level, ctypes.byref(nx), ctypes.byref(ny)), "grid_level_size")
    return nx.value, ny.value


def create_operator(g: int, omega2: float, hx: float, hy: float, hz: float, lambda2=1.0):
    """lambda2: a scalar, or a host array of shape (ny, nx) (lambda^2 per column)."""
    import numpy as np
    h = _P()
    col = None
    lam = 0.0
    if np.ndim(lambda2) == 0:
        lam = float(lambda2)
    else:
        col = np.ascontiguousarray(lambda2, dtype=np.float64)
    ptr = col.ctypes.data_as(_P) if col is not None else None
    _check(load().tpmg_create_operator(g, omega2, hx, hy, hz, lam, ptr, ctypes.byref(h)), "create_operator")
    return h.value


def destroy_operator(op: int) -> None:
    load().tpmg_destroy_operator(op)


def op_reserve(op: int, prec: int) -> None:
    _check(load().tpmg_op_reserve(op, prec), "op_reserve")


def op_level_coefficients(op: int, level: int, ncol: int):
    import numpy as np
    cx, cy = _D(), _D()
    v = np.empty(ncol)
    _check(load().tpmg_op_level_coefficients(op, level, ctypes.byref(cx), ctypes.byref(cy),
                                             v.ctypes.data_as(_P)), "op_level_coefficients")
    return cx.value, cy.value, v


# ---------------------------------------------------------------- single applications
def apply_A(op, level, prec, x, y, n, stream=None):
    _check(load().tpmg_apply_A(op, level, prec, _field(x, prec, n, "x"), _field(y, prec, n, "y"),
                               _stream(stream)), "apply_A")


def line_solve(op, level, prec, b, x, n, stream=None):
    _check(load().tpmg_line_solve(op, level, prec, _field(b, prec, n, "b"), _field(x, prec, n, "x"),
                                  _stream(stream)), "line_solve")


def smooth(op, level, prec, rho, u, f, u_out, n, norm_out=None, stream=None):
    _check(load().tpmg_smooth(op, level, prec, rho, _field(u, prec, n, "u"), _field(f, prec, n, "f"),
                              _field(u_out, prec, n, "u_out"), _scalar_out(norm_out), _stream(stream)),
           "smooth")


def residual(op, level, prec, u, f, r, n, norm_out=None, stream=None):
    _check(load().tpmg_residual(op, level, prec, _field(u, prec, n, "u"), _field(f, prec, n, "f"),
                                _field(r, prec, n, "r"), _scalar_out(norm_out), _stream(stream)), "residual")


def restrict_smooth(op, level, prec, rho, r_fine, f_c, u_c, n_fine, n_coarse, stream=None):
    _check(load().tpmg_restrict_smooth(op, level, prec, rho, _field(r_fine, prec, n_fine, "r_fine"),
                                       _field(f_c, prec, n_coarse, "f_c"), _field(u_c, prec, n_coarse, "u_c"),
                                       _stream(stream)), "restrict_smooth")


def residual_restrict_smooth(op, level, prec, rho, u_fine, f_fine, f_c, u_c, n_fine, n_coarse, stream=None):
    _check(load().tpmg_residual_restrict_smooth(op, level, prec, rho, _field(u_fine, prec, n_fine, "u_fine"),
                                                _field(f_fine, prec, n_fine, "f_fine"),
                                                _field(f_c, prec, n_coarse, "f_c"), _field(u_c, prec, n_coarse, "u_c"),
                                                _stream(stream)), "residual_restrict_smooth")


# every callback pair ever installed stays referenced: blocks it allocated go back to it later
_installed_allocators: list = []


def set_allocator(alloc, free) -> None:
    """Install Python callables as the library's device allocator: alloc(nbytes) -> device address
    (int, 256-byte aligned) or 0, free(address). None, None restores cudaMalloc / cudaFree."""
    if alloc is None and free is None:
        _check(load().tpmg_set_allocator(ALLOC_FN(), FREE_FN(), None), "set_allocator")
        return

    def _alloc(nbytes, ctx):
        try:
            return int(alloc(int(nbytes))) or None
        except Exception:  # reported by the library as TPMG_ERR_OOM
            return None

    def _free(ptr, ctx):
        free(int(ptr))

    pair = (ALLOC_FN(_alloc), FREE_FN(_free))
    _installed_allocators.append(pair)
    _check(load().tpmg_set_allocator(pair[0], pair[1], None), "set_allocator")


def use_torch_allocator(device=None) -> None:
    """Serve the library's device buffers from PyTorch's caching allocator (on `device`, default the
    current one): the library's workspace then shows in torch.cuda.memory_allocated()."""
    dev = torch.cuda.current_device() if device is None else device
    set_allocator(lambda n: torch.cuda.caching_allocator_alloc(n, dev), torch.cuda.caching_allocator_delete)


def use_cuda_allocator() -> None:
    set_allocator(None, None)


def set_fusion(op, enable) -> None:
    _check(load().tpmg_set_fusion(op, 1 if enable else 0), "set_fusion")


def prolongate(op, level, prec, u_c, u_f, n_coarse, n_fine, stream=None):
    _check(load().tpmg_prolongate(op, level, prec, _field(u_c, prec, n_coarse, "u_c"),
                                  _field(u_f, prec, n_fine, "u_f"), _stream(stream)), "prolongate")


def cg_fused_spmv(op, prec, alpha, beta, u, p, z, q, sigma_out, n, stream=None):
    _check(load().tpmg_cg_fused_spmv(op, prec, alpha, beta, _field(u, prec, n, "u"), _field(p, prec, n, "p"),
                                     _field(z, prec, n, "z"), _field(q, prec, n, "q"), _scalar_out(sigma_out),
                                     _stream(stream)), "cg_fused_spmv")


def cg_fused_tridiag(op, prec, alpha, r, q, z, rr_out, rz_out, n, stream=None):
    _check(load().tpmg_cg_fused_tridiag(op, prec, alpha, _field(r, prec, n, "r"), _field(q, prec, n, "q"),
                                        _field(z, prec, n, "z"), _scalar_out(rr_out), _scalar_out(rz_out),
                                        _stream(stream)), "cg_fused_tridiag")


# ---------------------------------------------------------------- solvers
def default_params(**kw) -> Params:
    p = Params()
    load().tpmg_default_params(ctypes.byref(p))
    names = {name for name, _ in Params._fields_}
    for k, v in kw.items():
        if k not in names:
            raise TypeError(f"unknown solver parameter {k!r}")
        if k == "prec" and isinstance(v, str):
            v = PREC[v]
        setattr(p, k, v)
    return p


def _solve(fn_name, op, params, f, u, n, history_len, stream, allow):
    prec = params.prec
    hist = (ctypes.c_double * max(history_len, 1))()
    info = Info()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    info.history_len = history_len
    status = getattr(load(), fn_name)(op, ctypes.byref(params), _field(f, prec, n, "f"),
                                      _field(u, prec, n, "u"), ctypes.byref(info), _stream(stream))
    _check(status, fn_name[5:], allow=allow)
    return {"status": status, "iters": info.iters, "converged": bool(info.converged),
            "rel_res": info.rel_res, "r0": info.r0, "ms": info.ms,
            "history": [hist[i] for i in range(min(info.iters + 1, history_len))]}


def mg_solve(op, params, f, u, n, history_len=256, stream=None, allow=(ERR_NOT_CONVERGED,)):
    return _solve("tpmg_mg_solve", op, params, f, u, n, history_len, stream, allow)


def mg_solve_mapped(op, params, f, u, n, history_len=256, stream=None, allow=(ERR_NOT_CONVERGED,)):
    """tpmg_mg_solve on page-locked host fields (CPU float64 tensors with is_pinned()) that the device
    addresses directly: the solve reads f and the initial u from the host and writes u back in its
    first and last kernels."""
    if params.prec not in (DW, MIXED):
        raise ValueError("host fields need prec DW or MIXED")
    for t, name in ((f, "f"), (u, "u")):
        if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.is_pinned() and t.dtype == torch.float64
                and t.is_contiguous() and t.numel() == n):
            raise TypeError(f"{name} must be a pinned contiguous CPU float64 tensor of {n} elements")
    hist = (ctypes.c_double * max(history_len, 1))()
    info = Info()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    info.history_len = history_len
    status = load().tpmg_mg_solve(op, ctypes.byref(params), f.data_ptr(), u.data_ptr(), ctypes.byref(info),
                                  _stream(stream))
    _check(status, "mg_solve", allow=allow)
    return {"status": status, "iters": info.iters, "converged": bool(info.converged),
            "rel_res": info.rel_res, "r0": info.r0, "ms": info.ms,
            "history": [hist[i] for i in range(min(info.iters + 1, history_len))]}


LAYOUT_X, LAYOUT_Z = 0, 1


def mg_solve_host(op, params, f, u, n, layout=LAYOUT_Z, history_len=256, stream=None, allow=(ERR_NOT_CONVERGED,)):
    """tpmg_mg_solve_host: f and u are CPU tensors (float64; float32 for F32) of n values in `layout`
    (LAYOUT_X: x fastest as on the device; LAYOUT_Z: z fastest, column by column); the library copies
    and transposes them on the device around the solve. Returns the solve's info plus "ms_io", the
    device time of the copies and transposes (info "ms" covers the whole call)."""
    dt = torch.float32 if params.prec == F32 else torch.float64
    for t, name in ((f, "f"), (u, "u")):
        if not (isinstance(t, torch.Tensor) and not t.is_cuda and t.dtype == dt and t.is_contiguous()
                and t.numel() == n):
            raise TypeError(f"{name} must be a contiguous CPU {dt} tensor of {n} elements")
    hist = (ctypes.c_double * max(history_len, 1))()
    info = Info()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    info.history_len = history_len
    ms_io = _D()
    status = load().tpmg_mg_solve_host(op, ctypes.byref(params), int(layout), f.data_ptr(), u.data_ptr(),
                                       ctypes.byref(info), ctypes.byref(ms_io), _stream(stream))
    _check(status, "mg_solve_host", allow=allow)
    return {"status": status, "iters": info.iters, "converged": bool(info.converged),
            "rel_res": info.rel_res, "r0": info.r0, "ms": info.ms, "ms_io": ms_io.value,
            "history": [hist[i] for i in range(min(info.iters + 1, history_len))]}


def cg_solve(op, params, f, u, n, history_len=4096, stream=None, allow=(ERR_NOT_CONVERGED,)):
    return _solve("tpmg_cg_solve", op, params, f, u, n, history_len, stream, allow)


def mg_solve_batched(ops, params, fs, us, history_len=128, stream=None, allow=(ERR_NOT_CONVERGED,)):
    """ops: list of operator handles; fs, us: lists of CUDA float64 fields (finest level of each)."""
    nb = len(ops)
    op_arr = (_P * nb)(*ops)
    f_arr = (_P * nb)(*[_field(f, F64, f.numel(), "f") for f in fs])
    u_arr = (_P * nb)(*[_field(u, F64, f.numel(), "u") for f, u in zip(fs, us)])
    infos = (Info * nb)()
    hists = [(ctypes.c_double * history_len)() for _ in range(nb)]
    for b in range(nb):
        infos[b].history = ctypes.cast(hists[b], ctypes.POINTER(ctypes.c_double))
        infos[b].history_len = history_len
    status = load().tpmg_mg_solve_batched(nb, ctypes.cast(op_arr, _P), ctypes.byref(params), ctypes.cast(f_arr, _P),
                                          ctypes.cast(u_arr, _P), ctypes.cast(infos, _P), _stream(stream))
    _check(status, "mg_solve_batched", allow=allow)
    return {"status": status, "ms": infos[0].ms,
            "problems": [{"iters": infos[b].iters, "converged": bool(infos[b].converged), "rel_res": infos[b].rel_res,
                          "r0": infos[b].r0, "history": [hists[b][i] for i in range(min(infos[b].iters + 1, history_len))]}
                         for b in range(nb)]}


def vcycle(op, params, f, u, n, stream=None):
    prec = params.prec
    _check(load().tpmg_vcycle(op, ctypes.byref(params), _field(f, prec, n, "f"), _field(u, prec, n, "u"),
                              _stream(stream)), "vcycle")


# ---------------------------------------------------------------- learned stage and flexible CG
def _f32(t, numel, name):
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
            and t.numel() == numel):
        raise TypeError(f"{name} must be a contiguous CUDA float32 tensor of {numel} elements")
    return t.data_ptr()


def nn_nparams(cin: int) -> int:
    return int(load().tpmg_nn_nparams(cin))


class Network:
    """Owns a tpmg_nn (the 4-layer convolutional preconditioner stage)."""

    def __init__(self, cin: int = 2, params=None):
        import numpy as np
        self.cin = cin
        self.nparams = nn_nparams(cin)
        h = _P()
        ptr = None
        if params is not None:
            self._init = np.ascontiguousarray(params, dtype=np.float32)
            assert self._init.size == self.nparams
            ptr = self._init.ctypes.data_as(_P)
        _check(load().tpmg_nn_create(cin, ptr, ctypes.byref(h)), "nn_create")
        self.h = h.value

    def get_params(self):
        import numpy as np
        out = np.empty(self.nparams, dtype=np.float32)
        _check(load().tpmg_nn_get_params(self.h, out.ctypes.data_as(_P)), "nn_get_params")
        return out

    def set_params(self, params):
        import numpy as np
        a = np.ascontiguousarray(params, dtype=np.float32)
        assert a.size == self.nparams
        _check(load().tpmg_nn_set_params(self.h, a.ctypes.data_as(_P)), "nn_set_params")

    def forward(self, x, shape, stream=None):
        nz, ny, nx = shape
        n = nx * ny * nz
        out = torch.empty(n, dtype=torch.float32, device=x.device)
        _check(load().tpmg_nn_forward(self.h, nx, ny, nz, _f32(x, n * self.cin, "x"), out.data_ptr(),
                                      _stream(stream)), "nn_forward")
        return out

    def loss_grad(self, x, target, shape, stream=None):
        nz, ny, nx = shape
        n = nx * ny * nz
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        grad = torch.empty(self.nparams, dtype=torch.float32, device=x.device)
        _check(load().tpmg_nn_loss_grad(self.h, nx, ny, nz, _f32(x, n * self.cin, "x"), _f32(target, n, "target"),
                                        loss.data_ptr(), grad.data_ptr(), _stream(stream)), "nn_loss_grad")
        return loss, grad

    def train_step(self, x, target, shape, lr, stream=None):
        nz, ny, nx = shape
        n = nx * ny * nz
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        _check(load().tpmg_nn_train_step(self.h, nx, ny, nz, _f32(x, n * self.cin, "x"), _f32(target, n, "target"),
                                         lr, loss.data_ptr(), _stream(stream)), "nn_train_step")
        return loss

    def loss_grad_residual(self, op, x, n, stream=None):
        """Residual loss mean((x0 - A D^-1 NN(x))^2), D = diag(A), on the finest level of the operator
        handle op (n cells)."""
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        grad = torch.empty(self.nparams, dtype=torch.float32, device=x.device)
        _check(load().tpmg_nn_loss_grad_residual(self.h, op, _f32(x, n * self.cin, "x"), loss.data_ptr(),
                                                 grad.data_ptr(), _stream(stream)), "nn_loss_grad_residual")
        return loss, grad

    def train_step_residual(self, op, x, n, lr, stream=None):
        loss = torch.zeros(1, dtype=torch.float64, device=x.device)
        _check(load().tpmg_nn_train_step_residual(self.h, op, _f32(x, n * self.cin, "x"), lr, loss.data_ptr(),
                                                  _stream(stream)), "nn_train_step_residual")
        return loss

    def close(self):
        if getattr(self, "h", None):
            load().tpmg_nn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nn_make_pair(op, shape, cin, r, u_star=None, u_k=None, aux=None, stream=None):
    """(x, target) for the network from a residual r and the error u_star - u_k (CUDA float64) on the
    finest level of the operator handle op (of the given (nz, ny, nx) shape)."""
    nz, ny, nx = shape
    n = nx * ny * nz
    x = torch.empty(n * cin, dtype=torch.float32, device=r.device)
    target = torch.empty(n, dtype=torch.float32, device=r.device) if u_star is not None else None
    _check(load().tpmg_nn_make_pair(op, cin, _field(r, F64, n, "r"),
                                    None if u_star is None else _field(u_star, F64, n, "u_star"),
                                    None if u_k is None else _field(u_k, F64, n, "u_k"),
                                    None if aux is None else _f32(aux, nx * ny, "aux"), x.data_ptr(),
                                    None if target is None else target.data_ptr(), _stream(stream)), "nn_make_pair")
    return x, target


def fcg_solve(op, params, f, u, n, nn=None, aux=None, history_len=512, stream=None, allow=(ERR_NOT_CONVERGED,)):
    hist = (ctypes.c_double * history_len)()
    info = Info()
    info.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
    info.history_len = history_len
    acc = _I(0)
    status = load().tpmg_fcg_solve(op, None if nn is None else nn.h,
                                   None if aux is None else aux.data_ptr(), ctypes.byref(params),
                                   _field(f, F64, n, "f"), _field(u, F64, n, "u"), ctypes.byref(info),
                                   ctypes.byref(acc), _stream(stream))
    _check(status, "fcg_solve", allow=allow)
    return {"status": status, "iters": info.iters, "converged": bool(info.converged), "rel_res": info.rel_res,
            "ms": info.ms, "nn_accepted": acc.value,
            "history": [hist[i] for i in range(min(info.iters + 1, history_len))]}


# ---------------------------------------------------------------- allocation-free variant
NOALLOC_MAX_BLOCKS = 65536


def residual_norm_noalloc(nx, ny, nz, cx, cy, v, u, f, r, norm_out, stream=None):
    """r = f - A u and ||r|| (FP64) for callers that must not allocate device memory: no operator,
    no workspace; the per-block partial sums live in the library's fixed device array. v is a CUDA
    float64 tensor of ny*nx vertical couplings; u, f, r are CUDA float64 fields; norm_out a CUDA
    float64 tensor of at least one element. Calls that overlap on the GPU must be serialised."""
    n = nx * ny * nz
    if not (isinstance(v, torch.Tensor) and v.is_cuda and v.dtype == torch.float64 and v.numel() == nx * ny
            and v.is_contiguous()):
        raise TypeError("v must be a contiguous CUDA float64 tensor of ny*nx elements")
    status = load().tpmg_residual_norm_noalloc(nx, ny, nz, cx, cy, v.data_ptr(), _field(u, F64, n, "u"),
                                               _field(f, F64, n, "f"), _field(r, F64, n, "r"),
                                               _scalar_out(norm_out), _stream(stream))
    if status != OK:
        raise TpmgError(status, "residual_norm_noalloc", load().tpmg_noalloc_last_error().decode())


# ---------------------------------------------------------------- profiling
def time_kernel(op, prec, kernel, reps=10, stream=None) -> float:
    """Mean duration in ms of one launch of an internal kernel on the operator's workspace."""
    ms = _D()
    _check(load().tpmg_time_kernel(op, prec, kernel, reps, ctypes.byref(ms), _stream(stream)), "time_kernel")
    return ms.value


def kernel_launches() -> int:
    return int(load().tpmg_kernel_launches())


ALU_FP64_FMA, ALU_FP64_ADD, ALU_FP64_MUL, ALU_FP32_FMA = range(4)


def measure_alu_rate(which: int, reps: int = 3) -> tuple[float, float]:
    """Measured arithmetic rate of the current GPU: (operations per second, ms per probe launch);
    a multiply-add counts as one operation."""
    rate, ms = _D(), _D()
    _check(load().tpmg_measure_alu_rate(which, reps, ctypes.byref(rate), ctypes.byref(ms)), "measure_alu_rate")
    return rate.value, ms.value


NUM_VARIANTS = 12


def autotune(op, prec, nlevels, reps=5, stream=None) -> list[int]:
    """Times the Smooth tile variants per level and keeps the fastest; returns [variant of level
    1, ..., variant of level L]."""
    out = (ctypes.c_int * (nlevels + 1))()
    _check(load().tpmg_autotune(op, prec, reps, ctypes.cast(out, _P), _stream(stream)), "autotune")
    return [out[l] for l in range(1, nlevels + 1)]


def set_variant(op, prec, level, variant) -> None:
    _check(load().tpmg_set_variant(op, prec, level, variant), "set_variant")


# ---------------------------------------------------------------- convenience owner object
# ---------------------------------------------------------------- the cubed-sphere panel operator
def create_panel_operator(g: int, omega2: float, lambda2: float, H: float, extent: float = 1.0):
    h = _P()
    _check(load().tpmg_create_panel_operator(g, omega2, lambda2, H, extent, ctypes.byref(h)), "create_panel_operator")
    return h.value


def panel_level_geometry(op, level, nx, ny):
    """(|T| (ny, nx), x-face coefficients (ny, nx + 1), y-face coefficients (ny + 1, nx)) as the
    library computed them."""
    import numpy as np
    area, ax, ay = np.empty((ny, nx)), np.empty((ny, nx + 1)), np.empty((ny + 1, nx))
    _check(load().tpmg_panel_level_geometry(op, level, area.ctypes.data_as(_P), ax.ctypes.data_as(_P),
                                            ay.ctypes.data_as(_P)), "panel_level_geometry")
    return area, ax, ay


def panel_apply_A(op, level, x, y, n, stream=None):
    _check(load().tpmg_panel_apply_A(op, level, _field(x, F64, n, "x"), _field(y, F64, n, "y"), _stream(stream)),
           "panel_apply_A")


def panel_line_solve(op, level, b, x, n, stream=None):
    _check(load().tpmg_panel_line_solve(op, level, _field(b, F64, n, "b"), _field(x, F64, n, "x"), _stream(stream)),
           "panel_line_solve")


def panel_smooth(op, level, rho, u, f, u_out, n, norm_out=None, stream=None):
    _check(load().tpmg_panel_smooth(op, level, rho, _field(u, F64, n, "u"), _field(f, F64, n, "f"),
                                    _field(u_out, F64, n, "u_out"), _scalar_out(norm_out), _stream(stream)),
           "panel_smooth")


def panel_residual(op, level, u, f, r, n, norm_out=None, stream=None):
    _check(load().tpmg_panel_residual(op, level, _field(u, F64, n, "u"), _field(f, F64, n, "f"),
                                      _field(r, F64, n, "r"), _scalar_out(norm_out), _stream(stream)),
           "panel_residual")


def panel_restrict_smooth(op, level, rho, r_fine, f_c, u_c, n_fine, n_coarse, stream=None):
    _check(load().tpmg_panel_restrict_smooth(op, level, rho, _field(r_fine, F64, n_fine, "r_fine"),
                                             _field(f_c, F64, n_coarse, "f_c"), _field(u_c, F64, n_coarse, "u_c"),
                                             _stream(stream)), "panel_restrict_smooth")


def panel_prolongate(op, level, u_c, u_f, n_coarse, n_fine, stream=None):
    _check(load().tpmg_panel_prolongate(op, level, _field(u_c, F64, n_coarse, "u_c"), _field(u_f, F64, n_fine, "u_f"),
                                        _stream(stream)), "panel_prolongate")


class PanelOperator:
    """Owns a grid and a cubed-sphere panel operator (native FP64)."""

    def __init__(self, nx, ny, nz, omega2, lambda2, H, extent=1.0, nlevels=0):
        self.grid = create_grid(nx, ny, nz, nlevels)
        self.op = None
        self.op = create_panel_operator(self.grid, omega2, lambda2, H, extent)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.L = grid_nlevels(self.grid)

    def level_shape(self, level):
        nx, ny = grid_level_size(self.grid, level)
        return (self.nz, ny, nx)

    def level_n(self, level):
        a, b, c = self.level_shape(level)
        return a * b * c

    def close(self):
        if self.op:
            destroy_operator(self.op)
            self.op = None
        if self.grid:
            destroy_grid(self.grid)
            self.grid = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Operator:
    """Owns a grid and an operator built from a workloads.Problem-like description."""

    def __init__(self, nx, ny, nz, omega2, hx, hy, hz, lambda2, nlevels=0):
        self.grid = create_grid(nx, ny, nz, nlevels)
        self.op = None
        self.op = create_operator(self.grid, omega2, hx, hy, hz, lambda2)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.L = grid_nlevels(self.grid)

    @classmethod
    def from_problem(cls, p, nlevels=None):
        return cls(p.nx, p.ny, p.nz, p.omega2, p.hx, p.hy, p.hz, p.lambda2,
                   p.nlevels if nlevels is None else nlevels)

    def level_shape(self, level):
        nx, ny = grid_level_size(self.grid, level)
        return (self.nz, ny, nx)

    def level_n(self, level):
        a, b, c = self.level_shape(level)
        return a * b * c

    def close(self):
        if self.op:
            destroy_operator(self.op)
            self.op = None
        if self.grid:
            destroy_grid(self.grid)
            self.grid = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
