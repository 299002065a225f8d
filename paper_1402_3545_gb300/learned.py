"""The learned preconditioner stage: training data from the multigrid solver, training, checkpoints
and its use in flexible CG. Every step runs in the CUDA library; this module only orders the calls.

The network answers in units of a Jacobi step: flexible CG adds s D^{-1} NN(r1/s) to its V-cycle
correction (s = rms(r1), D = diag(A)), so NN's outputs are O(1) for every mesh width and lambda^2.
(Without D^{-1} they would be O(1/D), about 1e-6 on the application grid: below what BF16 weights
moved by Adam steps of 1e-3 resolve.)

Training pairs. A problem is drawn with lambda^2 log-uniform in [1e2, 1e4] on a 256 x 256 x 64
grid with the horizontal mesh width of the grid the network is applied to (the pairs are periodic
crops of that regime: same c_x, c_y and the same range of vertical couplings), coarsened down to
1 x 1 columns (levels_full). Its reference solution u* is the mixed-precision multigrid solution
to relative residual 1e-10. From u_0 = 0, k = 1, 2, 3 FP64 V-cycles give iterates u_k; each yields
    x = r_k / rms(r_k) (plus, for two-channel networks, log10(lambda^2) - 3 per column),
    target = D (u* - u_k) / rms(r_k),     r_k = f - A u_k,
so the network learns the map from a multigrid residual to the error that remains, which is what
flexible CG asks of it after its own V-cycle (the residual r1 there has the same history).
Two losses, both means over cells, minimised by Adam:
    "error":    (NN(x) - target)^2, the error in the network's units;
    "residual": (x0 - A D^{-1} NN(x))^2, the residual the correction leaves. Flexible CG keeps a
                learned correction only when it lowers the residual norm; an error-trained
                network whose remaining error is rich in high frequencies fails that test, so the
                residual loss trains for the quantity the test compares.
"""
from __future__ import annotations

import dataclasses
import json
import time

import numpy as np
import torch

from . import tpmg, workloads


@dataclasses.dataclass
class TrainConfig:
    nx: int = 256
    ny: int = 256
    nz: int = 64
    h: float = 1.0 / 2048  # horizontal mesh width of the application grid
    hz: float = 1.0 / 64
    omega2: float = 1e-2
    lam_lo: float = 1e2
    lam_hi: float = 1e4
    n_problems: int = 16
    ks: tuple = (1, 2, 3)
    cin: int = 2
    steps: int = 600
    lr: float = 1e-3
    lr_final: float = 1e-4  # cosine decay to this rate
    tol_star: float = 1e-10
    loss: str = "residual"  # "error": mean (NN(x) - target)^2; "residual": mean (x0 - A NN(x))^2
    seed: int = 0

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


def aux_field(lambda2, nx: int, ny: int) -> torch.Tensor:
    """Second input channel: log10(lambda^2) - 3 per column (0 at lambda^2 = 1e3), CUDA fp32."""
    lam = np.broadcast_to(np.asarray(lambda2, dtype=np.float64), (ny, nx))
    return torch.from_numpy(np.ascontiguousarray(np.log10(lam) - 3.0).astype(np.float32).ravel()).cuda()


def levels_full(nx: int, ny: int) -> int:
    """Levels when halving both sides while both are even and the shorter one exceeds 1. A crop at
    the application grid's mesh width coarsened this far ends with the same c_x, c_y as the
    application grid's coarsest level (8 x 8 there): the crop's V-cycle then behaves like the
    top of the application's, where coarsening the crop only to 8 x 8 would leave a coarsest
    level with c_x in the tens that two smoothing steps cannot solve."""
    L = 1
    while nx % 2 == 0 and ny % 2 == 0 and min(nx, ny) > 1:
        nx //= 2
        ny //= 2
        L += 1
    return L


def generate_pairs(cfg: TrainConfig, log=None):
    """List of (x, target, lambda2, operator) on the GPU: len(ks) pairs per problem; the operator
    (a tpmg.Operator of the problem) is kept for the residual loss."""
    rng = np.random.default_rng(cfg.seed)
    nz, ny, nx = cfg.shape
    n = nx * ny * nz
    L = levels_full(nx, ny)
    pairs = []
    for i in range(cfg.n_problems):
        lam2 = float(10.0 ** rng.uniform(np.log10(cfg.lam_lo), np.log10(cfg.lam_hi)))
        op = tpmg.Operator(nx, ny, nz, cfg.omega2, cfg.h, cfg.h, cfg.hz, lam2, L)
        f = torch.from_numpy(workloads.make_rhs(nx, ny, nz, cfg.seed * 100003 + i, "uniform")).cuda()
        ustar = torch.zeros(n, dtype=torch.float64, device="cuda")
        res = tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.MIXED, tol=cfg.tol_star, max_iter=200), f, ustar, n)
        if not res["converged"]:
            raise RuntimeError(f"reference solve did not converge (lambda^2 = {lam2:.3g})")
        prm = tpmg.default_params(prec=tpmg.F64)
        u = torch.zeros(n, dtype=torch.float64, device="cuda")
        r = torch.empty(n, dtype=torch.float64, device="cuda")
        aux = aux_field(lam2, nx, ny) if cfg.cin == 2 else None
        done = 0
        for k in range(1, max(cfg.ks) + 1):
            tpmg.vcycle(op.op, prm, f, u, n)
            if k not in cfg.ks:
                continue
            tpmg.residual(op.op, op.L, tpmg.F64, u, f, r, n)
            x, t = tpmg.nn_make_pair(op.op, cfg.shape, cfg.cin, r, ustar, u, aux)
            pairs.append((x, t, lam2, op))
            done += 1
        if log:
            log(f"problem {i}: lambda^2 = {lam2:.3g}, reference in {res['iters']} iterations, {done} pairs")
    return pairs


def train(cfg: TrainConfig, pairs=None, net=None, log=None):
    """Adam on the pairs (one pair per step, drawn at random); returns (net, losses, seconds)."""
    if pairs is None:
        pairs = generate_pairs(cfg, log)
    if net is None:
        net = tpmg.Network(cfg.cin, init_params(cfg.cin, cfg.seed))
    rng = np.random.default_rng(cfg.seed + 1)
    losses = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    dev_losses = []
    n = cfg.nx * cfg.ny * cfg.nz
    for step in range(cfg.steps):
        x, t, _, op = pairs[int(rng.integers(len(pairs)))]
        lr = cfg.lr_final + 0.5 * (cfg.lr - cfg.lr_final) * (1.0 + np.cos(np.pi * step / max(cfg.steps, 1)))
        if cfg.loss == "residual":
            dev_losses.append(net.train_step_residual(op.op, x, n, lr))
        else:
            dev_losses.append(net.train_step(x, t, cfg.shape, lr))
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    losses = [float(l.item()) for l in dev_losses]
    if log:
        log(f"{cfg.steps} Adam steps in {secs:.2f} s; loss {np.mean(losses[:20]):.4g} -> {np.mean(losses[-20:]):.4g}")
    return net, losses, secs


def init_params(cin: int, seed: int) -> np.ndarray:
    """He-normal weights, zero biases; the last layer scaled by 0.1 so the first corrections are
    small (a fresh network is mostly rejected by the fallback rather than harmful)."""
    rng = np.random.default_rng(seed + 7)
    parts = []
    for i, (ci, co) in enumerate(((cin, 16), (16, 16), (16, 16), (16, 1))):
        w = np.sqrt(2.0 / (27 * ci)) * rng.standard_normal(co * ci * 27)
        parts.append(w * (0.1 if i == 3 else 1.0))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def evaluate(net, pairs, shape) -> dict:
    """Mean losses over pairs relative to the zero correction (no update): "error" =
    mean (NN(x) - target)^2 / mean target^2, "residual" = mean (x0 - A D^-1 NN(x))^2 / mean x0^2.
    A relative residual below 1 is a correction the flexible-CG test would keep."""
    n = int(np.prod(shape))
    err = res = 0.0
    for x, t, _, op in pairs:
        le, _ = net.loss_grad(x, t, shape)
        lr_, _ = net.loss_grad_residual(op.op, x, n)
        cin = x.numel() // n
        x0 = x.view(n, cin)[:, 0]
        err += float(le.item()) / float((t.double() ** 2).mean().item())
        res += float(lr_.item()) / float((x0.double() ** 2).mean().item())
    k = max(len(pairs), 1)
    return {"error": err / k, "residual": res / k}


def save(path: str, net, cfg: TrainConfig, extra: dict | None = None) -> None:
    meta = dataclasses.asdict(cfg)
    meta["ks"] = list(cfg.ks)
    if extra:
        meta.update(extra)
    np.savez(path, params=net.get_params(), cin=np.int32(net.cin), meta=np.array(json.dumps(meta)))


def load(path: str):
    """(Network, metadata dict) from a checkpoint written by save()."""
    z = np.load(path, allow_pickle=False)
    net = tpmg.Network(int(z["cin"]), z["params"].astype(np.float32))
    return net, json.loads(str(z["meta"]))


def fcg_compare(p: workloads.Problem, net=None, tol: float = 1e-6, max_iter: int = 200, reps: int = 1,
                solutions: dict | None = None):
    """Flexible CG with and without the learned stage on one problem (zero initial guess):
    iterations, device ms (median of reps), accepted corrections and the final relative residual.
    With a dict as `solutions`, each variant's final iterate is also stored there (host numpy)."""
    op = tpmg.Operator.from_problem(p)
    n = p.n
    f = torch.from_numpy(p.rhs()).cuda()
    aux = aux_field(p.lambda2, p.nx, p.ny) if net is not None and net.cin == 2 else None
    prm = tpmg.default_params(tol=tol, max_iter=max_iter)
    out = {}
    for name, nn in (("fcg_vcycle", None), ("fcg_learned", net)):
        if name == "fcg_learned" and net is None:
            continue
        ms = []
        for _ in range(reps):
            u = torch.zeros(n, dtype=torch.float64, device="cuda")
            res = tpmg.fcg_solve(op.op, prm, f, u, n, nn=nn, aux=aux)
            ms.append(res["ms"])
        out[name] = {"iters": res["iters"], "ms": float(np.median(ms)), "converged": res["converged"],
                     "rel_res": res["rel_res"], "nn_accepted": res["nn_accepted"]}
        if solutions is not None:
            solutions[name] = u.cpu().numpy()
    op.close()
    return out


def main(argv=None) -> None:
    """Train a network on generated pairs, report its losses and save a checkpoint."""
    import argparse
    ap = argparse.ArgumentParser(description="train the learned preconditioner stage")
    ap.add_argument("--out", required=True, help="checkpoint path (.npz)")
    ap.add_argument("--problems", type=int, default=TrainConfig.n_problems)
    ap.add_argument("--steps", type=int, default=TrainConfig.steps)
    ap.add_argument("--loss", choices=["residual", "error"], default=TrainConfig.loss)
    ap.add_argument("--cin", type=int, choices=[1, 2], default=TrainConfig.cin)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    cfg = TrainConfig(n_problems=a.problems, steps=a.steps, loss=a.loss, cin=a.cin, seed=a.seed)
    pairs = generate_pairs(cfg, log=print)
    held_out = generate_pairs(dataclasses.replace(cfg, n_problems=2, seed=cfg.seed + 1000))
    net, losses, secs = train(cfg, pairs, log=print)
    ev = evaluate(net, held_out, cfg.shape)
    print(f"held-out relative losses: {ev}")
    save(a.out, net, cfg, {"train_seconds": secs, "held_out": ev})


if __name__ == "__main__":
    main()
