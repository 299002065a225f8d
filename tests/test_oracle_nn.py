"""Pins of the learned-stage and flexible-CG oracle (no GPU): the convolution against torch's CPU
conv3d with circular/zero padding, gradients against torch autograd and central finite
differences, Adam against torch.optim.Adam, and flexible CG(1) with a fixed SPD preconditioner
against preconditioned CG (they coincide in exact arithmetic)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
from helpers import affine_network, assemble, rel, spectral_solve


def torch_conv(x, W, b):
    """x: (cin, nz, ny, nx) -> circular in x, y, zero in z, then a plain 3x3x3 correlation."""
    t = torch.as_tensor(x)[None]
    t = F.pad(t, (1, 1, 1, 1, 0, 0), mode="circular")
    t = F.pad(t, (0, 0, 0, 0, 1, 1))
    return F.conv3d(t, torch.as_tensor(W), None if b is None else torch.as_tensor(b))[0]


def rnd(shape, seed, scale=1.0):
    return scale * np.random.default_rng(seed).standard_normal(shape)


@pytest.mark.parametrize("cin,cout", [(2, 16), (16, 16), (16, 1), (3, 5)])
def test_conv3d_matches_torch(cin, cout):
    x = rnd((cin, 5, 6, 7), 1)
    W = rnd((cout, cin, 3, 3, 3), 2, 0.2)
    b = rnd((cout,), 3)
    y = oracle.conv3d(x, W, b)
    ref = torch_conv(x, W, b).numpy()
    assert rel(y, ref) < 1e-13
    yr = oracle.conv3d(x, W, b, relu=True)
    assert np.array_equal(yr, np.maximum(y, 0.0))


def test_conv3d_backward_matches_autograd():
    x = torch.tensor(rnd((3, 4, 5, 6), 4), requires_grad=True)
    W = torch.tensor(rnd((4, 3, 3, 3, 3), 5, 0.3), requires_grad=True)
    b = torch.tensor(rnd((4,), 6), requires_grad=True)
    dy = rnd((4, 4, 5, 6), 7)
    t = F.pad(F.pad(x[None], (1, 1, 1, 1, 0, 0), mode="circular"), (0, 0, 0, 0, 1, 1))
    y = F.conv3d(t, W, b)[0]
    (y * torch.as_tensor(dy)).sum().backward()
    dx, dW, db = oracle.conv3d_backward(x.detach().numpy(), W.detach().numpy(), dy)
    assert rel(dx, x.grad.numpy()) < 1e-12
    assert rel(dW, W.grad.numpy()) < 1e-12
    assert rel(db, b.grad.numpy()) < 1e-12


def _params(cin, seed):
    return rnd((oracle.nn_nparams(cin),), seed, 0.15)


def test_network_gradient_matches_finite_differences():
    """Central differences on a tiny grid; step 1e-6 in FP64 gives ~1e-9 relative accuracy."""
    cin = 2
    p = _params(cin, 8)
    x = rnd((cin, 4, 5, 6), 9)
    target = rnd((4, 5, 6), 10)
    loss, g = oracle.nn_loss_grad(p, x, target)
    rng = np.random.default_rng(11)
    for idx in rng.choice(p.size, size=25, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += h
        pm[idx] -= h
        num = (oracle.nn_loss_grad(pp, x, target)[0] - oracle.nn_loss_grad(pm, x, target)[0]) / (2 * h)
        assert abs(num - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])) + 1e-9, (idx, num, g[idx])


def _operator(nx, ny, seed):
    rng = np.random.default_rng(seed)
    return 3.0, 2.0, rng.uniform(5.0, 50.0, (ny, nx))


def test_residual_loss_gradient_matches_finite_differences():
    cin = 2
    p = _params(cin, 12)
    x = rnd((cin, 4, 5, 6), 13)
    cx, cy, v = _operator(6, 5, 14)
    loss, g = oracle.nn_loss_grad_residual(p, x, cx, cy, v)
    # the loss is what its definition says, with D taken from the assembled matrix's diagonal
    shape = x.shape[1:]
    D = np.diag(assemble(lambda a: oracle.apply_A(a, cx, cy, v), shape)).reshape(shape)
    assert np.allclose(oracle.diag_inv(shape, cx, cy, v), 1.0 / D, rtol=1e-15, atol=0)
    y = oracle.nn_forward(p, x) / D
    assert abs(loss - np.mean((x[0] - oracle.apply_A(y, cx, cy, v)) ** 2)) < 1e-12 * loss
    rng = np.random.default_rng(15)
    for idx in rng.choice(p.size, size=25, replace=False):
        h = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += h
        pm[idx] -= h
        num = (oracle.nn_loss_grad_residual(pp, x, cx, cy, v)[0] - oracle.nn_loss_grad_residual(pm, x, cx, cy, v)[0]) / (2 * h)
        assert abs(num - g[idx]) <= 1e-6 * max(1.0, abs(g[idx])) + 1e-9, (idx, num, g[idx])


def test_residual_loss_with_identity_operator_is_the_error_loss():
    """cx = cy = v = 0 leaves A = D = I: the residual loss is the error loss with target x[0]."""
    cin = 2
    p = _params(cin, 16)
    x = rnd((cin, 3, 4, 5), 17)
    l1, g1 = oracle.nn_loss_grad_residual(p, x, 0.0, 0.0, np.zeros((4, 5)))
    l2, g2 = oracle.nn_loss_grad(p, x, x[0])
    assert abs(l1 - l2) < 1e-14 * l2 and rel(g1, g2) < 1e-13


def test_network_forward_and_gradient_match_autograd():
    cin = 2
    p = _params(cin, 12)
    x = rnd((cin, 4, 6, 8), 13)
    target = rnd((4, 6, 8), 14)
    sizes = [16 * cin * 27, 16, 16 * 16 * 27, 16, 16 * 16 * 27, 16, 16 * 27, 1]
    shapes = [(16, cin, 3, 3, 3), (16,), (16, 16, 3, 3, 3), (16,), (16, 16, 3, 3, 3), (16,), (1, 16, 3, 3, 3), (1,)]
    pt = torch.tensor(p, requires_grad=True)
    chunks, off = [], 0
    for s, sh in zip(sizes, shapes):
        chunks.append(pt[off:off + s].reshape(sh))
        off += s
    h = torch.tensor(x)
    for layer in range(4):
        t = F.pad(F.pad(h[None], (1, 1, 1, 1, 0, 0), mode="circular"), (0, 0, 0, 0, 1, 1))
        h = F.conv3d(t, chunks[2 * layer], chunks[2 * layer + 1])[0]
        if layer < 3:
            h = torch.relu(h)
    out = h[0]
    assert rel(oracle.nn_forward(p, x), out.detach().numpy()) < 1e-12
    loss_t = ((out - torch.tensor(target)) ** 2).mean()
    loss_t.backward()
    loss, g = oracle.nn_loss_grad(p, x, target)
    assert abs(loss - loss_t.item()) < 1e-12 * loss
    assert rel(g, pt.grad.numpy()) < 1e-11


def test_adam_matches_torch():
    theta = rnd((50,), 15)
    th_t = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([th_t], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    for t in range(1, 4):
        g = rnd((50,), 16 + t)
        oracle.adam_step(theta, g, m, v, t, lr=1e-2)
        opt.zero_grad()
        th_t.grad = torch.tensor(g)
        opt.step()
    assert rel(theta, th_t.detach().numpy()) < 1e-12


def _problem():
    nx, ny, nz = 16, 16, 8
    cx = cy = 4.2 ** 2
    v = 1e-2 * 1e3 * nz ** 2
    f = rnd((nz, ny, nx), 20)
    return f, cx, cy, v


def test_fcg_with_fixed_spd_preconditioner_is_pcg():
    """FCG(1) with the fixed line-solve preconditioner reproduces textbook PCG's iteration."""
    f, cx, cy, v = _problem()
    _, it_cg, h_cg, c1 = oracle.cg_solve(f, cx, cy, v, tol=1e-8, max_iter=500)
    _, it_f, h_f, c2, _, _ = oracle.fcg_solve(f, cx, cy, v, mode=0, tol=1e-8, max_iter=500)
    assert c1 and c2 and abs(it_cg - it_f) <= 1
    k = min(15, it_cg)
    assert np.allclose(h_f[:k], h_cg[:k], rtol=1e-7)


def test_fcg_with_vcycle_converges_to_exact_solution():
    f, cx, cy, v = _problem()
    u, it, h, conv, _, _ = oracle.fcg_solve(f, cx, cy, v, mode=1, nlevels=2, tol=1e-11, max_iter=200)
    assert conv
    assert rel(u, spectral_solve(f, cx, cy, v)) < 1e-9
    # a V-cycle preconditioner beats the line solve by a wide margin
    _, it0, _, _, _, _ = oracle.fcg_solve(f, cx, cy, v, mode=0, tol=1e-11, max_iter=500)
    assert it < it0 / 2


def test_learned_stage_with_zero_network_always_falls_back():
    """A zero network proposes no correction, which never cuts the residual: every application is
    rejected and FCG proceeds exactly as with the plain V-cycle."""
    f, cx, cy, v = _problem()
    zero = np.zeros(oracle.nn_nparams(1))
    _, it1, h1, _, _, _ = oracle.fcg_solve(f, cx, cy, v, mode=1, nlevels=2, tol=1e-9)
    _, it2, h2, _, used, rejected = oracle.fcg_solve(f, cx, cy, v, mode=2, nlevels=2, tol=1e-9, params=zero)
    assert it1 == it2 and np.array_equal(h1, h2)
    # one application before the loop and one after every iteration but the last
    assert used == 0 and rejected == it2


def test_affine_network_is_affine():
    p = affine_network(2, 0.3, -0.7)
    x = rnd((2, 4, 5, 6), 30)
    assert np.allclose(oracle.nn_forward(p, x), 0.3 * x[0] - 0.7, rtol=0, atol=1e-15)


@pytest.mark.parametrize("alpha,beta", [(0.125, 0.0), (0.5, 1e-3), (0.125, -2e-3)])
def test_learned_candidate_by_hand(alpha, beta):
    """The learned candidate of one preconditioner application with the affine network, derived
    here from the V-cycle, the operator and the definitions: z1 = V(r), r1 = r - A z1,
    s = ||r1|| / sqrt(n), D = diag(A) read off the assembled matrix,
    c = z1 + s D^-1 (alpha r1/s + beta) = z1 + alpha D^-1 r1 + beta s D^-1 (a damped Jacobi step plus
    a constant), kept iff ||r - A c|| < ||r1||. The term beta s D^-1 is where the residual
    normalisation shows: a 2-norm reading instead of the root-mean-square one changes it by
    sqrt(n)."""
    f, cx, cy, v = _problem()
    n = f.size
    D = np.diag(assemble(lambda a: oracle.apply_A(a, cx, cy, v), f.shape)).reshape(f.shape)
    z1 = oracle.vcycle(np.zeros_like(f), f, cx, cy, v, 2)
    r1 = f - oracle.apply_A(z1, cx, cy, v)
    s = np.linalg.norm(r1) / np.sqrt(n)
    c = z1 + alpha * r1 / D + beta * s / D
    keep = np.linalg.norm(f - oracle.apply_A(c, cx, cy, v)) < np.linalg.norm(r1)
    z, cand, kept = oracle.fcg_precondition(f, cx, cy, v, mode=2, nlevels=2, params=affine_network(1, alpha, beta))
    assert rel(cand, c) < 1e-13
    assert kept == keep
    assert rel(z, c if keep else z1) < 1e-13


def test_learned_stage_first_step_by_hand():
    """One FCG step from u = 0: u1 = (<z, f> / <z, A z>) z with z the preconditioner's output
    (the damped-Jacobi candidate alpha = 1/8, which lowers the residual and is kept)."""
    f, cx, cy, v = _problem()
    p = affine_network(1, 0.125, 0.0)
    z, _, kept = oracle.fcg_precondition(f, cx, cy, v, mode=2, nlevels=2, params=p)
    assert kept
    u1 = (np.vdot(z, f) / np.vdot(z, oracle.apply_A(z, cx, cy, v))) * z
    u, it, _, _, used, rejected = oracle.fcg_solve(f, cx, cy, v, mode=2, nlevels=2, tol=1e-300, max_iter=1,
                                                   params=p)
    assert it == 1 and (used, rejected) == (1, 0)
    assert rel(u, u1) < 1e-12
