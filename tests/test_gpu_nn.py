"""The learned stage on the GPU against the oracle: the network's forward pass, its loss and
parameter gradient, Adam, and the training-pair builder, all through the C ABI.

The kernels keep weights, inputs and hidden activations in BF16 and accumulate in FP32. The oracle
runs in FP64 on the same BF16-rounded weights and inputs, so what separates the two is the
rounding of the three hidden activations (relative 2^-9 each) and of the data gradients in the
backward pass. Tolerances, relative 2-norm: output 2e-2 (three roundings of 2^-9 that add in
quadrature, times a cancellation factor of a few at the 16-channel sums); loss 2e-2; parameter
gradients 5e-2 (a fourth and fifth BF16 rounding on the data gradients). A network built to be
affine (helpers.affine_network) has no rounding after its input, so its output is held to FP32
accuracy."""
import numpy as np
import pytest
import torch

import oracle
from helpers import affine_network, rel
from paper_1402_3545_gb300 import tpmg

pytestmark = pytest.mark.gpu

SHAPES = [(3, 4, 64), (5, 6, 128), (1, 2, 64)]  # (nz, ny, nx): several tiles, odd nz, nz = 1


def bf16(a) -> np.ndarray:
    return torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).double().numpy()


def random_params(cin, seed, scale=1.0):
    """He-initialised weights and small biases (flat, the C ABI's layout)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in ((cin, 16), (16, 16), (16, 16), (16, 1)):
        parts.append(scale * np.sqrt(2.0 / (27 * ci)) * rng.standard_normal(co * ci * 27))
        parts.append(0.1 * rng.standard_normal(co))
    p = np.concatenate(parts).astype(np.float32)
    assert p.size == tpmg.nn_nparams(cin)
    return p


def weights_bf16(p, cin):
    """The parameters as the kernels use them: weights rounded to BF16, biases kept in FP32."""
    q = np.asarray(p, dtype=np.float64).copy()
    o = 0
    for ci, co in ((cin, 16), (16, 16), (16, 16), (16, 1)):
        q[o:o + co * ci * 27] = bf16(q[o:o + co * ci * 27])
        o += co * ci * 27 + co
    return q


def channels_last(x):
    """(cin, nz, ny, nx) -> flat CUDA fp32 tensor, cin values per cell."""
    return torch.from_numpy(np.ascontiguousarray(np.moveaxis(x, 0, -1)).astype(np.float32).ravel()).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.double().cpu().numpy()


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("cin", [1, 2])
def test_forward_matches_oracle(shape, cin):
    p = random_params(cin, seed=cin)
    x = np.random.default_rng(7).standard_normal((cin,) + shape)
    net = tpmg.Network(cin, p)
    y = host(net.forward(channels_last(x), shape)).reshape(shape)
    ref = oracle.nn_forward(weights_bf16(p, cin), bf16(x))
    assert rel(y, ref) < 2e-2, rel(y, ref)
    assert np.max(np.abs(y - ref)) < 5e-2 * np.max(np.abs(ref))
    net.close()


def _layers(params, cin):
    """(W, b) of the four layers from the flat parameters (W[co][ci][tap], tap = (dz, dy, dx))."""
    q = np.asarray(params, dtype=np.float64)
    out, o = [], 0
    for ci, co in ((cin, 16), (16, 16), (16, 16), (16, 1)):
        out.append((q[o:o + co * ci * 27].reshape(co, ci, 3, 3, 3), q[o + co * ci * 27:o + co * ci * 27 + co]))
        o += co * ci * 27 + co
    return out


def _forward_bf16_storage(params, x, cin):
    """The network with the GPU's storage: the oracle's layers (oracle.conv3d, FP64 sums) on
    BF16-rounded weights and input, every hidden activation rounded to BF16 after its ReLU, the
    output kept. Returns the output and the stored activations [x, a1, a2, a3]."""
    acts = [bf16(x)]
    for li, (W, b) in enumerate(_layers(weights_bf16(params, cin), cin)):
        y = oracle.conv3d(acts[-1], W, b, relu=li < 3)
        if li < 3:
            acts.append(bf16(y))
    return y[0], acts


# Layer-by-layer tolerances. With the GPU's BF16 storage reproduced, what remains is the FP32
# accumulation of each output's 27 * 16 = 432 products (relative ~sqrt(432) * 2^-24 ~ 1.2e-6, times a
# cancellation factor of up to ~10) and, where that difference straddles a BF16 rounding boundary,
# a stored value one BF16 ulp (2^-8 relative) away: a fraction ~1e-5 / 2^-8 ~ 3e-3 of the values, so
# ~sqrt(3e-3) * 2^-8 ~ 2e-4 relative per stored layer, ~4e-4 after three. Forward: 1e-3. Gradients
# go through five stored layers and parameter sums over every cell with cancellation: 1e-2. A slip in
# one layer's indexing, taps or channels is an O(1) error at either tolerance.
FWD_TOL, GRAD_TOL = 1e-3, 1e-2


# Shapes with nx % 128 = 0 and ny % 4 = 0 run every layer on the tensor-memory kernels (the 16 -> 16
# and last layers with tiles of 8 x 128 cells where ny % 8 = 0 and there are enough tiles to fill the
# SMs, else 4 x 128). (3, 700, 128): 175 tiles of 4 rows, more than the blocks, so blocks take tile
# pairs and some a lone last tile; (2, 2440, 128): 305 tiles of 8 rows (the last layer too, two
# blocks per SM), so some blocks run more than one; (1, 4, 128) and (2, 8, 256): one and two planes
# (the output plane completes after the last input plane; halo cells wrap to the tile's own other
# edge); (4, 12, 384): three tile columns, three tile rows.
ROLL_SHAPES = [(3, 700, 128), (2, 2440, 128), (1, 4, 128), (2, 8, 256), (4, 12, 384)]


@pytest.mark.parametrize("shape", SHAPES + ROLL_SHAPES, ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("cin", [1, 2])
def test_forward_matches_oracle_layers_with_bf16_storage(shape, cin):
    p = random_params(cin, seed=30 + cin)
    x = np.random.default_rng(31).standard_normal((cin,) + shape)
    # the layer composition itself, without rounding, is the oracle's network
    plain = x
    for li, (W, b) in enumerate(_layers(weights_bf16(p, cin), cin)):
        plain = oracle.conv3d(plain, W, b, relu=li < 3)
    assert rel(plain[0], oracle.nn_forward(weights_bf16(p, cin), x)) < 1e-13
    net = tpmg.Network(cin, p)
    y = host(net.forward(channels_last(x), shape)).reshape(shape)
    ref, _ = _forward_bf16_storage(p, x, cin)
    assert rel(y, ref) < FWD_TOL, rel(y, ref)
    net.close()


# (3, 8, 128): the data gradient of the 16 -> 16 layers on 4-row tiles; (2, 1216, 128): on 8-row
# tiles (152 of them), through the masked epilogue
@pytest.mark.parametrize("shape", SHAPES[:2] + [(3, 8, 128), (2, 1216, 128)], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("cin", [1, 2])
def test_gradient_matches_oracle_layers_with_bf16_storage(shape, cin):
    """Backpropagation as the kernels store it: the output gradient 2 (y - t) / n in FP32, every
    hidden data gradient (the ReLU mask times the transposed convolution of the next layer's) rounded
    to BF16; each layer's parameter gradient is the oracle's (oracle.conv3d_backward) on the stored
    input activations and the stored output gradient. Compared per weight and bias block."""
    p = random_params(cin, seed=40 + cin)
    rng = np.random.default_rng(41)
    x = rng.standard_normal((cin,) + shape)
    target = rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    y, acts = _forward_bf16_storage(p, x, cin)
    n = y.size
    layers = _layers(weights_bf16(p, cin), cin)
    d = (2.0 * (y - target) / n)[None]  # gradient of the output, (1, nz, ny, nx)
    grads = [None] * 4
    for li in (3, 2, 1, 0):
        W, _ = layers[li]
        dx, dW, db = oracle.conv3d_backward(acts[li], W, d, want_dx=li > 0)
        grads[li] = (dW, db)
        if li > 0:
            d = bf16(np.where(acts[li] > 0, dx, 0.0))
    net = tpmg.Network(cin, p)
    loss, grad = net.loss_grad(channels_last(x), torch.from_numpy(target.astype(np.float32).ravel()).cuda(), shape)
    loss, grad = float(host(loss)[0]), host(grad)
    assert abs(loss - np.mean((y - target) ** 2)) < FWD_TOL * loss
    o = 0
    for li, (ci, co) in enumerate(((cin, 16), (16, 16), (16, 16), (16, 1))):
        dW, db = grads[li]
        for size, ref, what in ((co * ci * 27, dW.ravel(), "W"), (co, db, "b")):
            g = grad[o:o + size]
            assert rel(g, ref) < GRAD_TOL, (what, li + 1, rel(g, ref))
            o += size
    net.close()


@pytest.mark.parametrize("cin", [1, 2])
def test_affine_network_is_exact(cin):
    """alpha * bf16(x0) + beta (+ gamma relu(bf16(x1))) to FP32 accuracy: the hidden layers only
    copy BF16 values, which BF16 holds exactly."""
    shape = (3, 4, 128)
    p = affine_network(cin, 2.0 ** -3, 0.37, gamma=0.5 if cin == 2 else 0.0).astype(np.float32)
    x = np.random.default_rng(8).standard_normal((cin,) + shape)
    net = tpmg.Network(cin, p)
    y = host(net.forward(channels_last(x), shape)).reshape(shape)
    xb = bf16(x)
    ref = 2.0 ** -3 * xb[0] + np.float32(0.37) + (0.5 * np.maximum(xb[1], 0.0) if cin == 2 else 0.0)
    assert np.max(np.abs(y - ref)) < 1e-6
    net.close()


@pytest.mark.parametrize("shape", SHAPES[:2], ids=lambda s: "x".join(map(str, s)))
@pytest.mark.parametrize("cin", [1, 2])
def test_loss_and_gradient_match_oracle(shape, cin):
    p = random_params(cin, seed=10 + cin)
    rng = np.random.default_rng(11)
    x = rng.standard_normal((cin,) + shape)
    target = rng.standard_normal(shape)
    net = tpmg.Network(cin, p)
    loss, grad = net.loss_grad(channels_last(x), torch.from_numpy(target.astype(np.float32).ravel()).cuda(), shape)
    loss, grad = float(host(loss)[0]), host(grad)
    ref_loss, ref_grad = oracle.nn_loss_grad(weights_bf16(p, cin), bf16(x), np.float32(target).astype(np.float64))
    assert abs(loss - ref_loss) < 2e-2 * ref_loss
    o = 0
    for ci, co in ((cin, 16), (16, 16), (16, 16), (16, 1)):
        for size, what in ((co * ci * 27, "W"), (co, "b")):
            g, r = grad[o:o + size], ref_grad[o:o + size]
            assert rel(g, r) < 5e-2, (what, ci, co, rel(g, r))
            o += size
    assert o == grad.size
    net.close()


@pytest.mark.parametrize("cin", [1, 2])
def test_residual_loss_and_gradient_match_oracle(cin):
    """mean((x0 - A NN(x))^2) with A the operator's finest level (FP32 on the GPU)."""
    from gpu_common import make_problem
    shape = (3, 4, 64)
    prob = make_problem(shape[2], shape[1], shape[0])
    op = tpmg.Operator.from_problem(prob, nlevels=1)
    cx, cy, v = oracle.problem_coefficients(prob)
    p = random_params(cin, seed=60 + cin, scale=0.3)
    x = np.random.default_rng(61).standard_normal((cin,) + shape)
    net = tpmg.Network(cin, p)
    loss, grad = net.loss_grad_residual(op.op, channels_last(x), prob.n)
    loss, grad = float(host(loss)[0]), host(grad)
    ref_loss, ref_grad = oracle.nn_loss_grad_residual(weights_bf16(p, cin), bf16(x), cx, cy, v)
    assert abs(loss - ref_loss) < 2e-2 * ref_loss, (loss, ref_loss)
    assert rel(grad, ref_grad) < 5e-2, rel(grad, ref_grad)
    net.close()
    op.close()


def test_adam_steps_match_oracle():
    """Three Adam steps on the GPU against the oracle's Adam fed with the GPU's own gradients:
    only the update rule is compared here (FP32 against FP64, relative 1e-5 of the step)."""
    cin, shape, lr = 2, (3, 4, 64), 1e-3
    p = random_params(cin, seed=20)
    rng = np.random.default_rng(21)
    x = channels_last(rng.standard_normal((cin,) + shape))
    target = torch.from_numpy(rng.standard_normal(shape).astype(np.float32).ravel()).cuda()
    net = tpmg.Network(cin, p)
    theta = p.astype(np.float64)
    m, v = np.zeros_like(theta), np.zeros_like(theta)
    for t in range(1, 4):
        _, g = net.loss_grad(x, target, shape)
        oracle.adam_step(theta, host(g), m, v, t, lr=lr)
        net.train_step(x, target, shape, lr)
        got = net.get_params().astype(np.float64)
        assert np.max(np.abs(got - theta)) < 1e-5 * lr * t + 1e-7 * np.max(np.abs(theta))
    net.close()


def test_training_reduces_the_loss():
    """Fitting a target the network can represent (a smoothed copy of its input) by Adam."""
    cin, shape = 1, (4, 8, 64)
    rng = np.random.default_rng(30)
    xin = rng.standard_normal((cin,) + shape)
    target = 0.5 * xin[0] + 0.25 * (np.roll(xin[0], 1, axis=2) + np.roll(xin[0], -1, axis=2))
    x = channels_last(xin)
    tt = torch.from_numpy(target.astype(np.float32).ravel()).cuda()
    net = tpmg.Network(cin, random_params(cin, seed=31, scale=0.5))
    first = float(host(net.train_step(x, tt, shape, 3e-3))[0])
    for _ in range(200):
        last = float(host(net.train_step(x, tt, shape, 3e-3))[0])
    assert last < 0.1 * first, (first, last)
    net.close()


@pytest.mark.parametrize("cin", [1, 2])
def test_make_pair(cin):
    """x = bf16(r / rms(r)) (and bf16(aux)), target = D (u* - u_k) / rms(r) with D = diag(A)."""
    from gpu_common import make_problem
    shape = (3, 4, 16)
    n = int(np.prod(shape))
    prob = make_problem(shape[2], shape[1], shape[0])
    op = tpmg.Operator.from_problem(prob, nlevels=1)
    cx, cy, v = oracle.problem_coefficients(prob)
    rng = np.random.default_rng(40)
    r, us, uk = (rng.standard_normal(shape) for _ in range(3))
    aux = rng.uniform(0.5, 2.0, shape[1:])
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a).ravel()).cuda()
    x, target = tpmg.nn_make_pair(op.op, shape, cin, d(r), d(us), d(uk),
                                  aux=d(aux.astype(np.float32)) if cin == 2 else None)
    rms = np.sqrt(np.sum(r * r) / n)
    x = host(x).reshape(shape + (cin,))
    ref0 = bf16(r / rms)
    # the scaled residual may round differently in its last FP32 bit: allow one BF16 step
    assert np.all(np.abs(x[..., 0] - ref0) <= 2.0 ** -7 * np.abs(ref0))
    if cin == 2:
        assert np.array_equal(x[..., 1], np.broadcast_to(bf16(aux.astype(np.float32)), shape))
    ref_t = (us - uk) / rms / oracle.diag_inv(shape, cx, cy, v)
    assert np.allclose(host(target).reshape(shape), ref_t, rtol=1e-6, atol=1e-7 * np.max(np.abs(ref_t)))
    op.close()


def test_shape_and_argument_errors():
    net = tpmg.Network(1)
    x = torch.zeros(2 * 4 * 96, dtype=torch.float32, device="cuda")
    with pytest.raises(tpmg.TpmgError):
        net.forward(x, (2, 4, 96))  # nx not a multiple of 64
    with pytest.raises(tpmg.TpmgError):
        net.forward(torch.zeros(3 * 64, dtype=torch.float32, device="cuda"), (1, 3, 64))  # odd ny
    with pytest.raises(tpmg.TpmgError):
        tpmg.Network(3)
    net.close()


def test_params_round_trip_and_zero_default():
    net = tpmg.Network(2)
    assert not np.any(net.get_params())
    p = random_params(2, seed=50)
    net.set_params(p)
    assert np.array_equal(net.get_params(), p)
    net.close()


def test_forward_full_size_sampled():
    """The forward pass at the learned workload's inference size, 2048^2 x 64 (every layer on 8-row
    tiles, several tiles per block, as the bench times it), against the oracle on sampled cells. An
    output depends on the input within 4 cells (four 3x3x3 layers), so the oracle evaluates each
    sampled cell on the 9^3 crop around it, wrapped in x and y and clipped at the z ends (where the
    network zero-pads): crop cells near the crop's own edges see wrong neighbours, but their errors
    move one cell inwards per layer and do not reach the centre in four. The samples include the
    volume's faces and corners and the edges of the 8 x 128 tiles."""
    nz, ny, nx, cin = 64, 2048, 2048, 2
    p = random_params(cin, seed=77)
    rng = np.random.default_rng(78)
    xl = rng.standard_normal((nz, ny, nx, cin), dtype=np.float32)  # channels-last, as the kernels read it
    net = tpmg.Network(cin, p)
    y = net.forward(torch.from_numpy(xl.reshape(-1)).cuda(), (nz, ny, nx))
    cells = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (0, ny - 1, 0), (nz - 1, 0, nx - 1), (1, 7, 127), (2, 8, 128),
             (31, 1023, 1024), (32, 1024, 1023), (62, 2047, 128), (63, 8, 2047)]
    cells += [tuple(int(v) for v in rng.integers(0, (nz, ny, nx))) for _ in range(30)]
    idx = torch.tensor([(k * ny + j) * nx + i for k, j, i in cells], device="cuda")
    got = y[idx].double().cpu().numpy()
    ref = np.empty(len(cells))
    for s, (k, j, i) in enumerate(cells):
        zlo, zhi = max(0, k - 4), min(nz, k + 5)
        crop = xl[zlo:zhi][:, np.arange(j - 4, j + 5) % ny][:, :, np.arange(i - 4, i + 5) % nx]
        yc, _ = _forward_bf16_storage(p, np.moveaxis(crop, -1, 0).astype(np.float64), cin)
        ref[s] = yc[k - zlo, 4, 4]
    assert rel(got, ref) < FWD_TOL, rel(got, ref)
    assert np.max(np.abs(got - ref)) < 1e-2 * np.max(np.abs(ref))
    net.close()
