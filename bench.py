#!/usr/bin/env python
"""Benchmark: multigrid solve time to a 1e-6 relative residual on the mid-size problem of the
paper's family (512 x 512 x 128 cells, lambda^2(x, y) varying, N(0,1) right-hand side, 7-level
V(2,2) tensor-product multigrid with vertical line smoothing), FP64-accurate arithmetic.

One step = one complete solve from a zero initial guess (every kernel of the multigrid path:
Smooth with fused residual norm, Residual, RestrictSmooth, Prolongate, the device-side
convergence test), inputs resident in HBM. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank solves its own copy of the problem:
the path has no data-parallel exchange, so ranks are independent replicas ("replicas only").
`--impl reference` times the oracle (plain FP64 C, test infrastructure) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_1402_3545_gb300 import workloads  # noqa: E402

METRIC = "MG solve ms to 1e-6 rel. residual & % of HBM peak, FP64 vs mixed/learned"
# dram__bytes_read.sum + dram__bytes_write.sum of one finest-level Smooth launch (k_sweep_x2,
# double-word) on the 512^2 x 128 problem, per tile variant, from the ncu captures summarised in
# profiles/k_sweep_x2_dw_smooth_mid_512x512x128.md (variant 6: 1.2650 GB + 0.3982 GB)
PROFILED_SMOOTH_TRAFFIC = {5: 1554562560, 6: 1663204352, 7: 1630302208}
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-only", action="store_true",
                    help="time the solves only (no kernel timing, e2e, variants or CPU baseline): "
                         "the command the ncu launch-list profile runs")
    ap.add_argument("--kernel-only", choices=["smooth", "residual", "restrict_smooth", "residual_restrict",
                                              "prolongate", "line_solve", "apply_A", "cg_spmv", "cg_tridiag",
                                              "nn_forward"],
                    help="launch only this finest-level kernel a few times (tile variant --variant, "
                         "no autotuning): the command a per-kernel ncu capture runs")
    ap.add_argument("--variant", type=int, default=3)
    ap.add_argument("--precision", choices=["dw", "f32", "f64"], default="dw")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def oracle_counts():
    path = os.path.join(ROOT, "tests", "golden", "oracle_counts.txt")
    out = {}
    if os.path.exists(path):
        for line in open(path):
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split(None, 1)
            out[k] = float(v)
    return out


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline_sample(p, f, iters_hint):
    """The oracle as it stands, on the host: one V-cycle and one residual on the full grid; the
    solve estimate is t_res + iters * (t_cycle + t_res) with the oracle's own iteration count."""
    import oracle
    cx, cy, v = oracle.problem_coefficients(p)
    u = np.zeros_like(f)
    t0 = time.perf_counter()
    r = oracle.residual(u, f, cx, cy, v)
    t_res = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.vcycle(u, f, cx, cy, v, p.nlevels)
    t_cycle = time.perf_counter() - t0
    del r
    counts = oracle_counts()
    iters = int(counts.get("mid_iters", iters_hint))
    est_ms = 1e3 * (t_res + iters * (t_cycle + t_res))
    return est_ms, {"t_cycle_s": round(t_cycle, 3), "t_residual_s": round(t_res, 3), "oracle_iters": iters}


def _oracle_replica(p, barrier, out):
    """One replica of the oracle sample in its own (spawned) process: the same residual and V-cycle
    on its own copy of the inputs, timed after every replica has its inputs ready."""
    import oracle
    f = p.rhs()
    cx, cy, v = oracle.problem_coefficients(p)
    u = np.zeros_like(f)
    barrier.wait(timeout=600)
    t0 = time.perf_counter()
    oracle.residual(u, f, cx, cy, v)
    t1 = time.perf_counter()
    oracle.vcycle(u, f, cx, cy, v, p.nlevels)
    out.put((t1 - t0, time.perf_counter() - t1))


def host_memory_bytes() -> int:
    """Memory this process may still use: MemAvailable, capped by a cgroup limit if one is set."""
    avail = 0
    with open("/proc/meminfo") as fh:
        for line in fh:
            if line.startswith("MemAvailable:"):
                avail = int(line.split()[1]) * 1024
    for path in ("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory/memory.limit_in_bytes"):
        try:
            raw = open(path).read().strip()
        except OSError:
            continue
        if raw.isdigit():
            used = 0
            for upath in ("/sys/fs/cgroup/memory.current", "/sys/fs/cgroup/memory/memory.usage_in_bytes"):
                try:
                    used = int(open(upath).read().strip())
                    break
                except (OSError, ValueError):
                    pass
            avail = min(avail, int(raw) - used)
    return avail


def cpu_baseline_all_cores(p, iters: int, bytes_per_replica: int):
    """The oracle on every host core at once: one replica of the single-core sample per core (as many
    as host memory allows at bytes_per_replica each), spawned processes, started together. Returns
    the per-solve time of the whole host (the slowest replica's solve estimate / replicas) and the
    details, or None when fewer than two replicas fit."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    fit = int(0.5 * host_memory_bytes() // bytes_per_replica)
    n = min(cores, fit)
    if n < 2:
        return None
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(n)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica, args=(p, barrier, out)) for _ in range(n)]
    for pr in procs:
        pr.start()
    res = []
    deadline = time.time() + 1200
    import queue
    while len(res) < n:
        try:
            res.append(out.get(timeout=2))
        except queue.Empty:
            # a replica that died (or a run past the deadline) ends the measurement
            if time.time() > deadline or any(pr.exitcode not in (None, 0) for pr in procs):
                for pr in procs:
                    if pr.is_alive():
                        pr.terminate()
                return None
    for pr in procs:
        pr.join(timeout=60)
    est = max(1e3 * (tr + iters * (tc + tr)) for tr, tc in res)
    return {"value": round(est / n, 3), "unit": "ms", "cores": n, "replicas": n,
            "slowest_replica_solve_ms": round(est, 3),
            "t_cycle_s_max": round(max(tc for _, tc in res), 3),
            "sample": (f"{n} concurrent replicas of the single-core sample (one process per core), "
                       f"slowest replica's solve estimate divided by {n}")}


def bench_batched(tpmg, torch):
    probs = workloads.batched()
    ops = [tpmg.Operator.from_problem(p) for p in probs]
    fs = [torch.from_numpy(p.rhs()).cuda() for p in probs]
    us = [torch.zeros_like(f) for f in fs]
    prm = tpmg.default_params(prec=tpmg.MIXED, tol=1e-6, max_iter=60)
    handles = [o.op for o in ops]
    for _ in range(2):
        for u in us:
            u.zero_()
        res = tpmg.mg_solve_batched(handles, prm, fs, us)
    times = []
    for _ in range(3):
        for u in us:
            u.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        res = tpmg.mg_solve_batched(handles, prm, fs, us)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    seq = []
    for _ in range(2):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for o, f, u, p in zip(ops, fs, us, probs):
            u.zero_()
            tpmg.mg_solve(o.op, prm, f, u, p.n)
        e1.record()
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
    out = {"ms": round(min(times), 3), "sequential_single_solves_ms": round(min(seq), 3),
           "problems": len(probs), "cells": int(sum(p.n for p in probs)),
           "all_converged": all(r["converged"] for r in res["problems"]),
           "iters_max": max(r["iters"] for r in res["problems"])}
    for o in ops:
        o.close()
    return out


def max_over_ranks(x: float, dist, device) -> float:
    """The largest of the ranks' values (every rank receives it); x itself on one process."""
    if not dist:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def per_solve_ms(elapsed_max_ms: float, steps: int, world: int) -> float:
    """Replicas only: every rank solves its own copy `steps` times, so the job solves steps * world
    problems in the slowest rank's time."""
    return elapsed_max_ms / (steps * world)


def cycle_memrefs(level_cells, nu_pre: int = 2, nu_post: int = 2, n_coarse: int = 2, smooth: float = 3,
                  residual: float = 3, restrict_smooth: float = 6, prolongate: float = 2.25, norm: float = 0,
                  fine_only: bool = False) -> float:
    """Memory references of one V(nu_pre, nu_post) cycle (Algorithm 1) from per-kernel costs per
    cell: on the finest level nu_pre + nu_post Smooths, a Residual, a Prolongate into it and the
    residual norm; on every coarser level but the coarsest a RestrictSmooth (the first pre-smoothing
    step, per cell of that level), nu_pre - 1 Smooths, a Residual, a Prolongate into it and nu_post
    Smooths; on the coarsest a RestrictSmooth and n_coarse - 1 Smooths. level_cells[l] = cells of
    level l (1 = coarsest .. L = finest; index 0 unused). fine_only: the finest level's share."""
    L = len(level_cells) - 1
    n = level_cells
    total = (smooth * (nu_pre + nu_post) + residual + prolongate + norm) * n[L]
    if fine_only:
        return total
    for l in range(2, L):
        total += (restrict_smooth + smooth * (nu_pre - 1) + residual + prolongate + smooth * nu_post) * n[l]
    total += (restrict_smooth + smooth * (n_coarse - 1)) * n[1]
    return total


def solve_memrefs(level_cells, iters: int, nu_pre: int = 2, nu_post: int = 2, n_coarse: int = 2) -> float:
    """Memory references of a whole multigrid solve by the minimal per-kernel model (Smooth and
    Residual 3 per cell -- the Thomas intermediates stay on chip --, RestrictSmooth 6 per coarse cell,
    Prolongate 2.25 per fine cell, the residual norm fused into the next Smooth): `iters` cycles plus
    the solve's first Smooth, which also yields the initial residual norm."""
    L = len(level_cells) - 1
    return 3 * level_cells[L] + iters * cycle_memrefs(level_cells, nu_pre, nu_post, n_coarse)


def nn_flops_per_voxel(cin: int) -> int:
    """Multiply-adds x 2 of the 4-layer network per voxel: 3x3x3 taps, cin -> 16 -> 16 -> 16 -> 1."""
    return 2 * 27 * (cin * 16 + 16 * 16 + 16 * 16 + 16)


def bench_mixed(tpmg, torch):
    """Mixed precision on its own workload (1024^2 x 128, lambda^2 = 1e4): FP32 V-cycles inside
    double-word refinement at 1e-6 and 1e-10, error against a 1e-12 double-word solution; also with
    the inner cycle's coarse levels holding BF16 values (coarse_bf16, a convergence measurement)."""
    p = workloads.mixed()
    op = tpmg.Operator.from_problem(p)
    f = torch.from_numpy(p.rhs()).cuda()
    n = p.n
    ustar = torch.zeros_like(f)
    tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.DW, tol=1e-12, max_iter=100), f, ustar, n)
    nrm = float(torch.linalg.vector_norm(ustar).item())
    out = {"workload": p.name}
    for name, prec, tol, bf in [("dw_1e-6", tpmg.DW, 1e-6, 0), ("mixed_1e-6", tpmg.MIXED, 1e-6, 0),
                                ("mixed_1e-10", tpmg.MIXED, 1e-10, 0),
                                ("mixed_1e-6_bf16_coarse", tpmg.MIXED, 1e-6, 1),
                                ("mixed_1e-10_bf16_coarse", tpmg.MIXED, 1e-10, 1)]:
        prm = tpmg.default_params(prec=prec, tol=tol, max_iter=100, coarse_bf16=bf)
        u = torch.zeros_like(f)
        ms = []
        for _ in range(3):
            u.zero_()
            r = tpmg.mg_solve(op.op, prm, f, u, n)
            ms.append(r["ms"])
        err = float(torch.linalg.vector_norm(u - ustar).item()) / nrm
        out[name] = {"ms": round(min(ms[1:]), 3), "iters": r["iters"], "rel_res": r["rel_res"],
                     "rel_err_vs_u_star": err}
    op.close()
    return out


def bench_paper_shaped(tpmg, torch):
    """The paper's own configuration on 512^2 x 128 (omega = 4.2 h, kappa ~ 142, lambda^2 = 1e3): V(1,1)
    multigrid with rho = 2/3 on 5 levels and line-preconditioned CG, both to 1e-5, FP64-accurate
    (double-word). The paper's figures on one K20X are context: 8 V-cycles of 88.8 ms, 59 CG
    iterations of 29.7 ms."""
    p = workloads.paper_shaped()
    op = tpmg.Operator.from_problem(p, nlevels=5)
    f = torch.from_numpy(p.rhs()).cuda()
    u = torch.zeros_like(f)
    out = {"workload": p.name}
    for name, fn, prm in [
            ("mg_v11", tpmg.mg_solve, tpmg.default_params(prec=tpmg.DW, tol=1e-5, max_iter=50, nu_pre=1, nu_post=1,
                                                          rho=2.0 / 3.0, zero_guess=1)),
            ("cg", tpmg.cg_solve, tpmg.default_params(prec=tpmg.DW, tol=1e-5, max_iter=500, zero_guess=1))]:
        ms = []
        for _ in range(3):
            r = fn(op.op, prm, f, u, p.n)
            ms.append(r["ms"])
        best = min(ms[1:])
        out[name] = {"ms": round(best, 3), "iters": r["iters"], "rel_res": r["rel_res"],
                     "ms_per_iter": round(best / max(r["iters"], 1), 4)}
    out["paper_k20x"] = {"mg_iters": 8, "ms_per_vcycle": 88.8, "cg_iters": 59, "ms_per_cg_iter": 29.7}
    op.close()
    return out


def bench_learned(tpmg, torch):
    """The learned stage: pairs from the multigrid solver on 256^2 x 64 crops, Adam on the residual
    loss, then flexible CG with and without the network on 2048^2 x 64 (h = 1/2048), beside plain
    double-word multigrid and the mixed solver, all to 1e-6."""
    from paper_1402_3545_gb300 import learned
    cfg = learned.TrainConfig(n_problems=8, steps=400)
    t0 = time.perf_counter()
    pairs = learned.generate_pairs(cfg)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    held = learned.generate_pairs(learned.TrainConfig(n_problems=2, seed=1000))
    net, losses, t_train = learned.train(cfg, pairs)
    ev = learned.evaluate(net, held, cfg.shape)
    vox = cfg.nx * cfg.ny * cfg.nz
    p = workloads.learned_target()
    x = torch.randn(p.n * cfg.cin, device="cuda", dtype=torch.float32)
    for _ in range(2):
        net.forward(x, (p.nz, p.ny, p.nx))
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        net.forward(x, (p.nz, p.ny, p.nx))
    e1.record()
    torch.cuda.synchronize()
    t_fwd = e0.elapsed_time(e1) / 3
    del x
    fl = nn_flops_per_voxel(cfg.cin)
    out = {"workload": p.name, "train": {
        "pairs": len(pairs), "pair_generation_s": round(t_pairs, 2), "steps": cfg.steps, "seconds": round(t_train, 2),
        "voxels_per_s": round(cfg.steps * vox / t_train, 1), "loss": cfg.loss,
        "first_loss": round(float(np.mean(losses[:10])), 5), "last_loss": round(float(np.mean(losses[-20:])), 5),
        "held_out_relative": {k: round(v, 5) for k, v in ev.items()}},
        "nn_forward": {"ms": round(t_fwd, 3), "flop_per_voxel": fl,
                       "tflops": round(fl * p.n / (t_fwd * 1e-3) / 1e12, 2)}}
    r = learned.fcg_compare(p, net, tol=1e-6, reps=2)
    out.update(r)
    op = tpmg.Operator.from_problem(p)
    f = torch.from_numpy(p.rhs()).cuda()
    for name, prec in [("mg_dw", tpmg.DW), ("mg_mixed", tpmg.MIXED)]:
        prm = tpmg.default_params(prec=prec, tol=1e-6, max_iter=100)
        u = torch.zeros_like(f)
        ms = []
        for _ in range(2):
            u.zero_()
            res = tpmg.mg_solve(op.op, prm, f, u, p.n)
            ms.append(res["ms"])
        out[name] = {"ms": round(min(ms), 3), "iters": res["iters"], "rel_res": res["rel_res"]}
    op.close()
    net.close()
    return out


def run_reference(args, rank, world):
    if rank != 0:  # replicas of the oracle would time the same host cores: rank 0 alone runs
        return
    p = workloads.mid()
    f = p.rhs()
    import oracle
    oracle.build()
    vals, info = [], None
    for s in range(args.warmup + args.steps):
        est, info = cpu_baseline_sample(p, f, 6)
        if s >= args.warmup:
            vals.append(est)
    value = float(np.mean(vals))
    sample = (f"one oracle V(2,2) cycle + one residual on the full {p.nx}x{p.ny}x{p.nz} grid per step, "
              f"scaled to a full solve with the oracle's iteration count ({info['oracle_iters']})")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nz": p.nz, "levels": p.nlevels,
                       "solver": "V(2,2), rho 0.8, 2 coarse steps", "tol": 1e-6},
            "cpu_baseline": {"value": round(value, 3), "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": sample, **info},
            "e2e": {"value": round(value, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_kernel_only(args):
    """A few launches of one finest-level kernel of the mid problem, for a profiler capture."""
    import torch
    from paper_1402_3545_gb300 import tpmg
    if args.kernel_only == "nn_forward":
        # the learned stage's forward pass on one 256^2 x 64 training crop (4.2 M voxels)
        from paper_1402_3545_gb300 import learned
        shape = (64, 256, 256)
        nvox = shape[0] * shape[1] * shape[2]
        net = tpmg.Network(2, learned.init_params(2, 0))
        x = torch.randn(nvox * 2, device="cuda", dtype=torch.float32, generator=torch.Generator("cuda").manual_seed(0))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        net.forward(x, shape)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(max(args.steps, 1)):
            net.forward(x, shape)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / max(args.steps, 1)
        print(json.dumps({"kernel": "nn_forward", "voxels": nvox, "ms_per_forward": round(ms, 4),
                          "tflops": round(nn_flops_per_voxel(2) * nvox / (ms * 1e-3) / 1e12, 2)}), flush=True)
        net.close()
        return
    prec = {"dw": tpmg.DW, "f32": tpmg.F32, "f64": tpmg.F64}[args.precision]
    kid = {"smooth": tpmg.K_SMOOTH, "residual": tpmg.K_RESIDUAL, "restrict_smooth": tpmg.K_RESTRICT_SMOOTH,
           "prolongate": tpmg.K_PROLONGATE, "line_solve": tpmg.K_LINE_SOLVE, "cg_spmv": tpmg.K_CG_SPMV,
           "cg_tridiag": tpmg.K_CG_TRIDIAG, "residual_restrict": tpmg.K_RESIDUAL_RESTRICT,
           "apply_A": tpmg.K_APPLY_A}[args.kernel_only]
    p = workloads.mid()
    op = tpmg.Operator.from_problem(p)
    tpmg.op_reserve(op.op, tpmg.MIXED if prec == tpmg.F32 else prec)
    for l in range(1, op.L + 1):
        tpmg.set_variant(op.op, prec, l, args.variant)
    ms = tpmg.time_kernel(op.op, prec, kid, reps=max(args.steps, 1))
    torch.cuda.synchronize()
    print(json.dumps({"kernel": args.kernel_only, "precision": args.precision, "variant": args.variant,
                      "workload": p.name, "ms_per_launch": round(ms, 4)}), flush=True)
    op.close()


def run_ours(args, rank, world, dist):
    import torch
    from paper_1402_3545_gb300 import tpmg

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = workloads.mid()
    f = p.rhs()
    n = p.n
    op = tpmg.Operator.from_problem(p)
    prec = tpmg.DW
    prm = tpmg.default_params(prec=prec, tol=1e-6, max_iter=100, zero_guess=1)
    tpmg.op_reserve(op.op, prec)
    from paper_1402_3545_gb300 import autotune
    variants_dw = autotune.tune(op, prec, lambda_varies=True)
    fd = torch.from_numpy(f).to(dev)
    u = torch.zeros_like(fd)
    stream = torch.cuda.current_stream()

    def solve():  # from u = 0 (zero_guess: the solve clears its own copy of u, u is output only)
        return tpmg.mg_solve(op.op, prm, fd, u, n)

    for _ in range(max(args.warmup, 3)):
        res = solve()
    assert res["converged"], res
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    smi_index = int(vis.split(",")[local]) if vis and vis.split(",")[local].isdigit() else local
    sampler = ClockSampler(smi_index)
    sampler.start()
    time.sleep(0.3)
    k0 = tpmg.kernel_launches()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    iters = []
    for _ in range(args.steps):
        res = solve()
        iters.append(res["iters"])
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    launches = tpmg.kernel_launches() - k0
    clocks = sampler.stop()
    elapsed = e0.elapsed_time(e1)
    elapsed = max_over_ranks(elapsed, dist, dev)
    ms_per_step = elapsed / args.steps
    value = per_solve_ms(elapsed, args.steps, world)
    if args.solve_only:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": round(value, 4), "unit": "ms", "iters": iters[-1],
                              "gpu_launches": int(launches), "solve_only": True}), flush=True)
        op.close()
        return

    # dominant kernel: the finest-level Smooth (4 of the 5 fine-level sweeps of each cycle)
    t_smooth = tpmg.time_kernel(op.op, prec, tpmg.K_SMOOTH, reps=20)
    peaks, peak_kind = measured_peaks()
    bytes_smooth = 3 * 8 * n  # read u, f; write u' (8-byte values)
    achieved = bytes_smooth / (t_smooth * 1e-3) / 1e9
    finest_variant = variants_dw[-1] if variants_dw else None
    kernel_ms = {name: round(tpmg.time_kernel(op.op, prec, kid, reps=10), 4) for name, kid in [
        ("residual", tpmg.K_RESIDUAL), ("restrict_smooth", tpmg.K_RESTRICT_SMOOTH),
        ("residual_restrict_fused", tpmg.K_RESIDUAL_RESTRICT), ("apply_A", tpmg.K_APPLY_A),
        ("prolongate", tpmg.K_PROLONGATE), ("cg_spmv", tpmg.K_CG_SPMV), ("cg_tridiag", tpmg.K_CG_TRIDIAG)]}
    kernel_ms["smooth"] = round(t_smooth, 4)
    tpmg.op_reserve(op.op, tpmg.MIXED)
    variants_f32 = autotune.tune(op, tpmg.F32, lambda_varies=True)
    kernel_ms_f32 = {name: round(tpmg.time_kernel(op.op, tpmg.F32, kid, reps=10), 4) for name, kid in [
        ("smooth", tpmg.K_SMOOTH), ("residual", tpmg.K_RESIDUAL), ("line_solve", tpmg.K_LINE_SOLVE),
        ("restrict_smooth", tpmg.K_RESTRICT_SMOOTH), ("residual_restrict_fused", tpmg.K_RESIDUAL_RESTRICT),
        ("prolongate", tpmg.K_PROLONGATE)]}
    # native FP64 Smooth against the FP64 ALU: per cell the stencil residual (3 FMAs and 4 adds),
    # the forward elimination (FMA and multiply), the back substitution (2 FMAs) and the norm (FMA)
    # are 12 FP64 operations; GB300's nominal FP64 rate is 1.25 TFLOP/s (0.625 T FMA-or-add/s)
    tpmg.op_reserve(op.op, tpmg.F64)
    t_smooth64 = tpmg.time_kernel(op.op, tpmg.F64, tpmg.K_SMOOTH, reps=5)
    ops64 = 12 * n
    roofline_f64 = {"bound": "alu", "kernel": "finest-level native FP64 Smooth", "unit": "T FP64 ops/s",
                    "achieved": round(ops64 / (t_smooth64 * 1e-3) / 1e12, 4), "peak": 0.625,
                    "frac": round(ops64 / (t_smooth64 * 1e-3) / 1e12 / 0.625, 4), "ms_per_launch": round(t_smooth64, 4),
                    "ops_per_launch": ops64, "peak_source": "nominal 1.25 TFLOP/s FP64 (FMA or add per op)",
                    "hbm_frac_same_launch": round(3 * 8 * n / (t_smooth64 * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}
    n_smooth = 4 * iters[-1] + 1
    # DRAM bytes of one launch from the ncu capture summarised in
    # profiles/k_sweep_x2_dw_smooth_mid_512x512x128.md (null for a variant without a capture)
    traffic = PROFILED_SMOOTH_TRAFFIC.get(finest_variant)
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": traffic,
                "kernel": f"finest-level double-word Smooth (tile variant {finest_variant})",
                "peak_source": peak_kind, "bytes_per_launch": bytes_smooth, "ms_per_launch": round(t_smooth, 4),
                "share_of_solve": round(n_smooth * t_smooth / ms_per_step, 3),
                # lambda^2 varies over the level, so the Thomas factors 1/m_k and v/m_k are read per cell
                "bytes_with_factors": 5 * 8 * n,
                "frac_with_factors": round(5 * 8 * n / (t_smooth * 1e-3) / 1e9 / peaks["hbm_gbs"], 4)}

    # the whole solve's useful bandwidth: the paper's per-kernel memory references x 8 B per solve
    # (double-word and native FP64 levels both store 8-byte values) over the solve time
    level_cells = [0] + [op.level_n(l) for l in range(1, op.L + 1)]
    solve_bytes = 8 * solve_memrefs(level_cells, iters[-1])
    solve_hbm = {"bytes_per_solve": int(solve_bytes), "ms_per_solve": round(value, 4),
                 "achieved": round(solve_bytes / (value * 1e-3) / 1e9, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": round(solve_bytes / (value * 1e-3) / 1e9 / peaks["hbm_gbs"], 4), "peak_source": peak_kind,
                 "model": ("memory references of the paper's kernels (Smooth and Residual 3 per cell, "
                           "RestrictSmooth 6 per coarse cell, Prolongate 2.25 per fine cell) x 8 B, "
                           f"{iters[-1]} V(2,2) cycles + the first Smooth; the fused Residual+RestrictSmooth "
                           "moves less than its two kernels' share")}

    # end to end through the public API with host buffers, two ways: (a) the solve reads f from
    # page-locked host memory and writes u back there in its first and last kernels; (b) explicit
    # copies around a device solve (H2D of f, solve, D2H of u). Both start from u = 0 (zero_guess)
    # and move 8 bytes per cell each way; the faster is reported.
    f_h = torch.from_numpy(f).pin_memory()
    u_h = torch.zeros_like(f_h).pin_memory()
    for _ in range(2):
        tpmg.mg_solve_host(op.op, prm, f_h, u_h, n)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        tpmg.mg_solve_host(op.op, prm, f_h, u_h, n)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_host_ms = e0.elapsed_time(e1) / args.steps
    for _ in range(2):
        fd.copy_(f_h, non_blocking=True)
        solve()
        u_h.copy_(u, non_blocking=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        fd.copy_(f_h, non_blocking=True)
        solve()
        u_h.copy_(u, non_blocking=True)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_copy_ms = e0.elapsed_time(e1) / args.steps
    if e2e_host_ms <= e2e_copy_ms:
        e2e_ms, e2e_path = e2e_host_ms, "tpmg_mg_solve on page-locked host f and u"
    else:
        e2e_ms, e2e_path = e2e_copy_ms, "cudaMemcpyAsync of f, tpmg_mg_solve on device fields, cudaMemcpyAsync of u"

    # error of each solution against u*, a double-word solve of the same problem to a 1e-12
    # relative residual (outside every timed region)
    ustar = torch.zeros_like(fd)
    tpmg.mg_solve(op.op, tpmg.default_params(prec=tpmg.DW, tol=1e-12, max_iter=100), fd, ustar, n)
    ustar_norm = float(torch.linalg.vector_norm(ustar).item())

    def err_vs_ustar(x):
        return float(torch.linalg.vector_norm(x - ustar).item()) / ustar_norm

    u.zero_()
    solve()
    headline_err = err_vs_ustar(u)

    # the other precisions on the same problem (one solve each, after a warm-up solve)
    variants = {}
    for name, vprec, tol, bf in [("f64_native", tpmg.F64, 1e-6, 0), ("mixed_fp32_inner", tpmg.MIXED, 1e-6, 0),
                                 ("mixed_fp32_inner_1e-10", tpmg.MIXED, 1e-10, 0),
                                 ("mixed_bf16_coarse", tpmg.MIXED, 1e-6, 1)]:
        vp = tpmg.default_params(prec=vprec, tol=tol, max_iter=100, coarse_bf16=bf)
        for _ in range(2):
            u.zero_()
            r = tpmg.mg_solve(op.op, vp, fd, u, n)
        variants[name] = {"ms": round(r["ms"], 3), "iters": r["iters"], "rel_res": r["rel_res"],
                          "rel_err_vs_u_star": err_vs_ustar(u)}
    u.zero_()
    r = tpmg.cg_solve(op.op, tpmg.default_params(prec=tpmg.DW, tol=1e-6, max_iter=5000), fd, u, n)
    variants["cg_dw"] = {"ms": round(r["ms"], 3), "iters": r["iters"], "rel_res": r["rel_res"],
                         "rel_err_vs_u_star": err_vs_ustar(u)}
    del ustar

    # batched workload: 64 problems of drawn sizes in one persistent launch vs one solve after another
    variants["batched_64"] = bench_batched(tpmg, torch)
    variants["mixed_1024x1024x128"] = bench_mixed(tpmg, torch)
    variants["paper_shaped_512x512x128"] = bench_paper_shaped(tpmg, torch)
    variants["learned_2048x2048x64"] = bench_learned(tpmg, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        est, info = cpu_baseline_sample(p, f, iters[-1])
        cpu = {"value": round(est, 3), "unit": "ms", "cores": 1, "kind": "oracle",
               "sample": (f"one oracle V(2,2) cycle + one residual on the full {p.nx}x{p.ny}x{p.nz} grid, "
                          f"scaled to a full solve with the oracle's iteration count"), **info}
        # the same sample on all host cores at once (replicas; peak about 10 FP64 fields each)
        allc = cpu_baseline_all_cores(p, info["oracle_iters"], 10 * 8 * p.n)
        if allc is not None:
            cpu["all_cores"] = allc

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "dw (FP64 storage, double-word fp32 pair arithmetic)", "data": "synthetic",
                "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nz": p.nz, "levels": op.L,
                           "solver": "V(2,2), rho 0.8, 2 coarse steps", "tol": 1e-6, "precision": "DW",
                           "parallelism": f"replicas{world}",
                           "l2": "inputs larger than L2 (268 MB per FP64 field > 129 MB)"},
                "iters": iters[-1], "rel_err_vs_u_star": headline_err,
                "roofline": roofline, "solve_hbm": solve_hbm, "roofline_f64": roofline_f64,
                "kernel_ms": kernel_ms,
                "kernel_ms_f32": kernel_ms_f32,
                "tile_variants": {"dw": variants_dw, "f32": variants_f32}, "variants": variants,
                "e2e": {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": 8 * n,
                        "d2h_bytes_per_step": 8 * n, "path": e2e_path,
                        "host_fields_ms": round(e2e_host_ms, 4), "explicit_copies_ms": round(e2e_copy_ms, 4)},
                "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": int(launches)}
        print(json.dumps(line), flush=True)
    op.close()


def main():
    args = parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.kernel_only:
        run_kernel_only(args)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        tdist.init_process_group("nccl")
        dist = tdist
    run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
