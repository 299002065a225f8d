"""The host-buffer solve (tpmg_mg_solve_host), the paper's "total solution time" path of Sec. 5.1:
fields in host memory, copied to the device and -- from the vertically contiguous layout of a CPU
code -- transposed there to the horizontally contiguous layout of Eq. (13), solved, transposed and
copied back. The transposes move values without arithmetic, so the result must equal the device
solve on the same problem bit for bit, in every precision and both layouts; the grid's column count
and nz are not multiples of the 32 x 32 transpose tile, so the ragged tile edges are exercised.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_common import host, make_problem
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu

PRECS = [tpmg.F64, tpmg.DW, tpmg.MIXED, tpmg.F32]
IDS = ["f64", "dw", "mixed", "f32"]


@pytest.fixture(scope="module")
def prob():
    p = make_problem(96, 72, 45)  # 6912 columns, nz = 45: neither a multiple of 32
    op = tpmg.Operator.from_problem(p)
    yield p, op, p.rhs()
    op.close()


def _zfast(a):
    return np.ascontiguousarray(np.asarray(a).transpose(1, 2, 0))  # (ny, nx, nz): column by column


@pytest.mark.parametrize("prec", PRECS, ids=IDS)
@pytest.mark.parametrize("layout", [tpmg.LAYOUT_X, tpmg.LAYOUT_Z], ids=["x", "z"])
@pytest.mark.parametrize("zero_guess", [1, 0], ids=["zero_guess", "u_in"])
def test_host_solve_equals_device_solve(prob, prec, layout, zero_guess):
    p, op, f = prob
    dt = torch.float32 if prec == tpmg.F32 else torch.float64
    u0 = 0.01 * np.random.default_rng(7).standard_normal(f.shape)
    prm = tpmg.default_params(prec=prec, tol=1e-8, max_iter=60, zero_guess=zero_guess)
    fd = torch.from_numpy(f).to("cuda", dt).reshape(-1)
    ud = torch.from_numpy(u0).to("cuda", dt).reshape(-1)
    rd = tpmg.mg_solve(op.op, prm, fd, ud, p.n)
    lay = (lambda a: a) if layout == tpmg.LAYOUT_X else _zfast
    fh = torch.from_numpy(lay(f)).to(dt).reshape(-1).pin_memory()
    uh = torch.from_numpy(lay(u0)).to(dt).reshape(-1).pin_memory()
    rh = tpmg.mg_solve_host(op.op, prm, fh, uh, p.n, layout=layout)
    assert rh["iters"] == rd["iters"] and rh["history"] == rd["history"]
    u_dev = host(ud).reshape(f.shape)
    u_host = uh.double().numpy()
    u_host = u_host.reshape(f.shape) if layout == tpmg.LAYOUT_X else u_host.reshape(p.ny, p.nx, p.nz).transpose(2, 0, 1)
    assert np.array_equal(u_host, u_dev)
    assert rh["ms"] >= rh["ms_io"] > 0.0


def test_host_solve_from_pageable_memory_matches_oracle(prob):
    """Pageable (not page-locked) host arrays in the vertically contiguous layout: the native FP64
    solve to 1e-8 agrees with the oracle's multigrid iterate to 1e-10 after the same number of cycles."""
    p, op, f = prob
    cx, cy, v = oracle.problem_coefficients(p)
    prm = tpmg.default_params(prec=tpmg.F64, tol=1e-8, max_iter=60, zero_guess=1)
    fh = torch.from_numpy(_zfast(f)).reshape(-1)
    uh = torch.zeros(p.n, dtype=torch.float64)
    rh = tpmg.mg_solve_host(op.op, prm, fh, uh, p.n, layout=tpmg.LAYOUT_Z)
    u_ref, it_ref, _, _ = oracle.mg_solve(f, cx, cy, v, p.nlevels, tol=1e-8, max_iter=60)
    assert rh["iters"] == it_ref
    u = uh.numpy().reshape(p.ny, p.nx, p.nz).transpose(2, 0, 1)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-10
