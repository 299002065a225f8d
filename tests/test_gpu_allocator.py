"""A caller-supplied device allocator (tpmg_set_allocator): with PyTorch's caching allocator
serving the library's buffers the solve is the same bit for bit, the buffers show in
torch.cuda.memory_allocated() while the operator lives and go back when it is destroyed."""
import pytest
import torch

from gpu_common import dev, make_problem
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu


def solve(p, f):
    op = tpmg.Operator.from_problem(p)
    try:
        u = torch.zeros_like(f)
        res = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.DW, tol=1e-8, max_iter=60), f, u, p.n)
        torch.cuda.synchronize()
        return res, u, op
    except Exception:
        op.close()
        raise


def test_torch_allocator_serves_the_library():
    p = make_problem(128, 128, 16)
    f = dev(p.rhs(), tpmg.F64)
    res0, u0, op0 = solve(p, f)
    op0.close()
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    tpmg.use_torch_allocator()
    try:
        res1, u1, op1 = solve(p, f)
        held = torch.cuda.memory_allocated() - before - u1.numel() * u1.element_size()
        op1.close()
        torch.cuda.synchronize()
        after = torch.cuda.memory_allocated() - u1.numel() * u1.element_size()
    finally:
        tpmg.use_cuda_allocator()
    assert res0["iters"] == res1["iters"] and res0["history"] == res1["history"]
    assert torch.equal(u0, u1)
    # the hierarchy alone holds several fields of the finest level
    assert held >= 4 * p.n * 8, held
    assert after <= before, (before, after)


def test_allocator_needs_both_functions():
    lib = tpmg.load()
    assert lib.tpmg_set_allocator(tpmg.ALLOC_FN(lambda n, c: None), tpmg.FREE_FN(), None) == tpmg.ERR_ARG
    assert lib.tpmg_set_allocator(tpmg.ALLOC_FN(), tpmg.FREE_FN(), None) == tpmg.OK
