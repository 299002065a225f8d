#!/usr/bin/env python
"""Benchmark: multigrid solve time to a 1e-6 relative residual on the mid-size problem of the
paper's family (512 x 512 x 128 cells, lambda^2(x, y) varying, N(0,1) right-hand side, 7-level
V(2,2) tensor-product multigrid with vertical line smoothing), in native FP64 arithmetic -- the
paper's precision -- beside the same solve in double-word and mixed FP32/FP64 arithmetic.

One step = one complete native-FP64 solve from a zero initial guess (every kernel of the multigrid
path: Smooth with fused residual norm, Residual + RestrictSmooth, Prolongate, the device-side
convergence test), inputs resident in HBM. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torch.distributed.run) every rank solves its own copy of the problem:
the path has no data-parallel exchange, so ranks are independent replicas ("replicas only").
`--impl reference` times the oracle (plain FP64 C, test infrastructure) on the host cores, one
complete solve per step. The CPU leg of the default run (rank 0, one GPU) times the oracle the same
way and measures every GPU solution against an independent reference: the oracle's own solve to
1e-12 for the varying-coefficient problem, the exact spectral solution for the constant ones.
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
HBM_FALLBACK_GBS = 6800.0
# DRAM bytes per launch from ncu captures, keyed by kernel, precision, tile variant and workload
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.txt")
# FP64 operations of one finest-level Smooth per cell (the timed launch also forms the norm):
# stencil residual 3 multiply-adds + 4 adds, elimination 1 multiply-add + 1 multiply, back
# substitution and update 2 multiply-adds, norm 1 multiply-add -> 12 instructions, 19 flops
SMOOTH_F64_INSTR, SMOOTH_F64_FLOPS = 12, 19


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--solve-only", action="store_true",
                    help="time the solves only (no kernel timing, e2e, variants or CPU leg): "
                         "the command the ncu launch-list profile runs")
    ap.add_argument("--solve-precision", choices=["f64", "dw", "mixed"], default="f64",
                    help="precision of the --solve-only solves")
    ap.add_argument("--kernel-only", choices=["smooth", "residual", "restrict_smooth", "residual_restrict",
                                              "prolongate", "line_solve", "apply_A", "cg_spmv", "cg_tridiag",
                                              "nn_forward", "alu_rate", "transpose", "panel_smooth"],
                    help="launch only this finest-level kernel a few times (tile variant --variant, "
                         "no autotuning): the command a per-kernel ncu capture runs; alu_rate prints "
                         "the measured FP64 and FP32 arithmetic rates")
    ap.add_argument("--variant", type=int, default=3)
    ap.add_argument("--nn-nx", type=int, default=256, help="horizontal size of the nn_forward kernel-only grid")
    ap.add_argument("--nn-ny", type=int, default=0, help="its y size (default: the x size)")
    ap.add_argument("--precision", choices=["dw", "f32", "f64"], default="dw")
    return ap.parse_args()


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d, "measured"
    return {"hbm_gbs": HBM_FALLBACK_GBS, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def read_traffic() -> dict:
    """{(kernel, precision, variant, workload): (bytes, source)} from the tracked ncu summary."""
    out = {}
    if os.path.exists(TRAFFIC_FILE):
        for line in open(TRAFFIC_FILE):
            parts = line.split()
            if len(parts) >= 5 and not line.startswith("#"):
                out[(parts[0], parts[1], int(parts[2]), parts[3])] = (int(parts[4]), " ".join(parts[5:]))
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


def cpu_model() -> str:
    """The host CPU's name from /proc/cpuinfo (x86: model name; Arm: implementer and part)."""
    info = {}
    try:
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                info.setdefault(k.strip(), v.strip())
    except OSError:
        return "unknown"
    if "model name" in info:
        return info["model name"]
    return f"implementer {info.get('CPU implementer', '?')} part {info.get('CPU part', '?')}"


def oracle_solve(p, f, threads: int, tol: float = 1e-6, max_iter: int = 100):
    """One complete oracle multigrid solve of problem p (V(2,2), rho 0.8, two coarse steps, from
    zero) on `threads` host threads: (u, cycles, seconds, threads used)."""
    import oracle
    cx, cy, v = oracle.problem_coefficients(p)
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    u, it, _, _ = oracle.mg_solve(f, cx, cy, v, p.nlevels, tol=tol, max_iter=max_iter)
    return u, it, time.perf_counter() - t0, used


def rel_err(u, ref) -> float:
    u = np.asarray(u, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    return float(np.linalg.norm(u - ref) / np.linalg.norm(ref))


def cpu_leg(p, f, sols: dict):
    """The CPU side of the default run: the oracle timed on the host cores (one complete solve on all
    of them, and one on a single core), then every GPU solution measured against an independent
    reference -- the oracle's own solve to 1e-12 for the varying-coefficient mid problem, the exact
    spectral solution (oracle.spectral) for the constant-coefficient mixed, learned and batched
    problems -- and the headline solution's residual recomputed by the oracle."""
    import oracle
    from oracle import spectral
    cores = os.cpu_count() or 1
    u_all, it_all, t_all, used = oracle_solve(p, f, cores)
    _, it1, t1, _ = oracle_solve(p, f, 1)
    cpu = {"value": round(1e3 * t_all, 1), "unit": "ms", "cores": used, "kind": "oracle",
           "sample": (f"one complete oracle solve of the {p.nx}x{p.ny}x{p.nz} problem to 1e-6 "
                      f"({it_all} V(2,2) cycles) on {used} host threads (OpenMP over columns)"),
           "oracle_iters": it_all, "cpu_model": cpu_model(),
           "one_core": {"value": round(1e3 * t1, 1), "unit": "ms", "cores": 1, "oracle_iters": it1}}
    del u_all
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    cx, cy, v = oracle.problem_coefficients(p)
    ustar, it_s, hist, _ = oracle.mg_solve(f, cx, cy, v, p.nlevels, tol=1e-12, max_iter=40)
    ref = {"mid": {"reference": f"oracle multigrid solve to {hist[-1]:.1e} ({it_s} cycles)",
                   "rel_err": {k: rel_err(u, ustar) for k, u in sols.pop("mid").items()}}}
    r = oracle.residual(sols["mid_headline_u"], f, cx, cy, v)
    ref["mid"]["headline_rel_res_by_oracle"] = float(np.linalg.norm(r) / np.linalg.norm(f))
    del ustar, r, sols["mid_headline_u"]
    for key, prob in (("mixed", workloads.mixed()), ("learned", workloads.learned_target())):
        if key not in sols:
            continue
        fx = prob.rhs()
        cxx, cyy, vv = oracle.problem_coefficients(prob)
        uex = spectral.exact_solve(fx, cxx, cyy, vv)
        ref[key] = {"reference": "exact spectral solution (Fourier x Fourier x DCT-II)",
                    "rel_err": {k: rel_err(u, uex) for k, u in sols.pop(key).items()}}
        del fx, uex
    if "panel" in sols:
        from oracle import panel as opanel
        pp = workloads.panel()
        ref_p = opanel.PanelProblem(pp.nx, pp.ny, pp.nz, pp.nlevels, pp.omega2, pp.lambda2, pp.H, pp.extent)
        fp = pp.rhs()
        up, itp, _, _ = ref_p.mg_solve(fp, tol=1e-5, max_iter=60, nu_pre=1, nu_post=1, rho=2.0 / 3.0)
        ug = sols.pop("panel").reshape(fp.shape)
        ref["panel"] = {"reference": f"the panel oracle's own solve ({itp} V(1,1) cycles to 1e-5)",
                        "rel_err": rel_err(ug, up),
                        "rel_res_by_oracle": float(np.linalg.norm(ref_p.residual(ug, fp)) / np.linalg.norm(fp))}
    if "batched" in sols:
        errs = []
        for prob, u in zip(workloads.batched(), sols.pop("batched")):
            cxx, cyy, vv = oracle.problem_coefficients(prob)
            errs.append(rel_err(u, spectral.exact_solve(prob.rhs(), cxx, cyy, vv)))
        ref["batched"] = {"reference": "exact spectral solution of each problem",
                          "rel_err_max": max(errs), "rel_err_median": float(np.median(errs))}
    ref["seconds"] = round(time.perf_counter() - t0, 1)
    return cpu, ref


def run_reference(args, rank, world):
    """The reference arm: the oracle as it stands, one complete solve of the mid problem per step on
    all host cores (OpenMP over columns). Rank 0 alone runs (replicas would time the same cores)."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    p = workloads.mid()
    f = p.rhs()
    cores = os.cpu_count() or 1
    vals, iters, used = [], 0, cores
    for s in range(args.warmup + args.steps):
        _, iters, secs, used = oracle_solve(p, f, cores)
        if s >= args.warmup:
            vals.append(1e3 * secs)
    value = float(np.mean(vals))
    sample = (f"one complete oracle solve of the {p.nx}x{p.ny}x{p.nz} problem to 1e-6 ({iters} V(2,2) cycles) "
              f"per step on {used} host threads (OpenMP over columns)")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(value, 3),
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nz": p.nz, "levels": p.nlevels,
                       "solver": "V(2,2), rho 0.8, 2 coarse steps", "tol": 1e-6},
            "cpu_baseline": {"value": round(value, 3), "unit": "ms", "cores": used, "kind": "oracle",
                             "sample": sample, "oracle_iters": iters, "cpu_model": cpu_model()},
            "e2e": {"value": round(value, 3), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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


def bench_batched(tpmg, torch, sols=None):
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
    if sols is not None:
        sols["batched"] = [u.cpu().numpy() for u in us]
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


def bench_mixed(tpmg, torch, sols=None):
    """The mixed-precision workload (1024^2 x 128, lambda^2 = 1e4): FP32 V-cycles inside double-word
    refinement at 1e-6 and 1e-10, beside native FP64 and double-word multigrid at 1e-6; also with the
    inner cycle's coarse levels holding BF16 values (coarse_bf16, a convergence measurement). Each
    solution's error against the exact spectral solution is measured in the CPU leg."""
    p = workloads.mixed()
    op = tpmg.Operator.from_problem(p)
    f = torch.from_numpy(p.rhs()).cuda()
    n = p.n
    out = {"workload": p.name}
    keep = {}
    for name, prec, tol, bf in [("f64_1e-6", tpmg.F64, 1e-6, 0), ("dw_1e-6", tpmg.DW, 1e-6, 0),
                                ("mixed_1e-6", tpmg.MIXED, 1e-6, 0), ("mixed_1e-10", tpmg.MIXED, 1e-10, 0),
                                ("mixed_1e-6_bf16_coarse", tpmg.MIXED, 1e-6, 1),
                                ("mixed_1e-10_bf16_coarse", tpmg.MIXED, 1e-10, 1)]:
        prm = tpmg.default_params(prec=prec, tol=tol, max_iter=100, coarse_bf16=bf, zero_guess=1)
        u = torch.zeros_like(f)
        ms = []
        for _ in range(3):
            r = tpmg.mg_solve(op.op, prm, f, u, n)
            ms.append(r["ms"])
        out[name] = {"ms": round(min(ms[1:]), 3), "iters": r["iters"], "rel_res": r["rel_res"]}
        if sols is not None and not bf:
            keep[name] = u.cpu().numpy()
    if sols is not None:
        sols["mixed"] = keep
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


def bench_robustness(tpmg, torch):
    """The robustness study of Sec. 5.2 on the paper's 512^2 x 128 grid: nu_CFL = 2 omega / h from
    0.84 to 840, multigrid V(1,1) (rho = 2/3, epsilon = 1e-5) with 5, 7 and 10 levels and the coarse
    smoothing steps the paper needed, and line-preconditioned CG, native FP64: cycles or iterations
    and device ms of each solve."""
    out = {"settings": "V(1,1), rho 2/3, tol 1e-5, native FP64; CG tol 1e-5"}
    for nu in workloads.ROBUSTNESS_CFL:
        row = {}
        for L in workloads.ROBUSTNESS_LEVELS:
            p = workloads.paper_shaped(nu_cfl=nu, nlevels=L)
            nc = workloads.robustness_coarse_steps(L, nu)
            op = tpmg.Operator.from_problem(p, nlevels=L)
            f = torch.from_numpy(p.rhs()).cuda()
            u = torch.zeros_like(f)
            prm = tpmg.default_params(prec=tpmg.F64, tol=1e-5, max_iter=300, nu_pre=1, nu_post=1, n_coarse=nc,
                                      rho=2.0 / 3.0, zero_guess=1)
            ms = []
            for _ in range(2):
                r = tpmg.mg_solve(op.op, prm, f, u, p.n)
                ms.append(r["ms"])
            row[f"mg_{L}_levels"] = {"iters": r["iters"], "converged": r["converged"], "ms": round(min(ms), 3),
                                     "coarse_steps": nc}
            if L == workloads.ROBUSTNESS_LEVELS[0]:
                r = tpmg.cg_solve(op.op, tpmg.default_params(prec=tpmg.F64, tol=1e-5, max_iter=20000, zero_guess=1),
                                  f, u, p.n)
                row["cg"] = {"iters": r["iters"], "converged": r["converged"], "ms": round(r["ms"], 3)}
            op.close()
        out[f"cfl_{nu:g}"] = row
    return out


def bench_panel(tpmg, torch, sols=None):
    """The paper's own operator (Eq. (1) on a gnomonic cubed-sphere panel, Eq. (14)) in its single-GPU
    configuration: 512^2 x 128, 5 levels, V(1,1), rho = 2/3, epsilon = 1e-5, native FP64 multigrid and
    line-preconditioned CG, and the mixed solver (FP64 outer residual, FP32 V-cycles) at 1e-5 and
    1e-10; the paper's figures on one K20X are context."""
    p = workloads.panel()
    op = tpmg.PanelOperator(p.nx, p.ny, p.nz, p.omega2, p.lambda2, p.H, p.extent, nlevels=p.nlevels)
    f = torch.from_numpy(p.rhs()).cuda().reshape(-1)
    u = torch.zeros_like(f)
    prm = tpmg.default_params(prec=tpmg.F64, tol=1e-5, max_iter=60, nu_pre=1, nu_post=1, rho=2.0 / 3.0, zero_guess=1)
    ms = []
    for _ in range(4):
        r = tpmg.mg_solve(op.op, prm, f, u, p.n)
        ms.append(r["ms"])
    best = min(ms[1:])
    if sols is not None:
        sols["panel"] = u.cpu().numpy()
    out = {"workload": p.name, "mg_v11_f64": {"ms": round(best, 3), "iters": r["iters"], "rel_res": r["rel_res"],
                                              "ms_per_cycle": round(best / max(r["iters"], 1), 4)}}
    cg_prm = tpmg.default_params(prec=tpmg.F64, tol=1e-5, max_iter=2000, zero_guess=1)
    ms = []
    for _ in range(2):
        r = tpmg.cg_solve(op.op, cg_prm, f, u, p.n)
        ms.append(r["ms"])
    out["cg_f64"] = {"ms": round(min(ms), 3), "iters": r["iters"], "rel_res": r["rel_res"],
                     "ms_per_iter": round(min(ms) / max(r["iters"], 1), 4)}
    for name, tol in [("mg_mixed", 1e-5), ("mg_mixed_1e-10", 1e-10)]:
        mprm = tpmg.default_params(prec=tpmg.MIXED, tol=tol, max_iter=80, nu_pre=1, nu_post=1, rho=2.0 / 3.0,
                                  zero_guess=1)
        ms = []
        for _ in range(3):
            r = tpmg.mg_solve(op.op, mprm, f, u, p.n)
            ms.append(r["ms"])
        out[name] = {"ms": round(min(ms[1:]), 3), "iters": r["iters"], "rel_res": r["rel_res"]}
    out["mg_mixed"]["speedup_vs_mg_v11_f64"] = round(best / out["mg_mixed"]["ms"], 3)
    out["paper_k20x"] = {"mg_iters": 8, "ms_per_vcycle": 88.8, "cg_iters": 59, "ms_per_cg_iter": 29.7}
    op.close()
    return out


def bench_learned(tpmg, torch, sols=None):
    """The learned stage: pairs from the multigrid solver on 256^2 x 64 crops, Adam on the residual
    loss, then flexible CG with and without the network on 2048^2 x 64 (h = 1/2048), beside native
    FP64, double-word and mixed multigrid, all to 1e-6."""
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
    keep = {} if sols is not None else None
    r = learned.fcg_compare(p, net, tol=1e-6, reps=2, solutions=keep)
    out.update(r)
    op = tpmg.Operator.from_problem(p)
    f = torch.from_numpy(p.rhs()).cuda()
    for name, prec in [("mg_f64", tpmg.F64), ("mg_dw", tpmg.DW), ("mg_mixed", tpmg.MIXED)]:
        prm = tpmg.default_params(prec=prec, tol=1e-6, max_iter=100, zero_guess=1)
        u = torch.zeros_like(f)
        ms = []
        for _ in range(2):
            res = tpmg.mg_solve(op.op, prm, f, u, p.n)
            ms.append(res["ms"])
        out[name] = {"ms": round(min(ms), 3), "iters": res["iters"], "rel_res": res["rel_res"]}
        if keep is not None:
            keep[name] = u.cpu().numpy()
    if sols is not None:
        sols["learned"] = keep
    op.close()
    net.close()
    return out


def run_kernel_only(args):
    """A few launches of one finest-level kernel of the mid problem, for a profiler capture; or the
    measured arithmetic rates (alu_rate); or one host-buffer solve's copies and transposes."""
    import torch
    from paper_1402_3545_gb300 import tpmg
    if args.kernel_only == "alu_rate":
        out = {"kernel": "alu_rate", "unit": "T operations/s (a multiply-add counts once)"}
        for name, which in [("fp64_fma", tpmg.ALU_FP64_FMA), ("fp64_add", tpmg.ALU_FP64_ADD),
                            ("fp64_mul", tpmg.ALU_FP64_MUL), ("fp32_fma", tpmg.ALU_FP32_FMA)]:
            rate, ms = tpmg.measure_alu_rate(which, reps=max(args.steps, 1))
            out[name] = round(rate / 1e12, 4)
            out[name + "_ms"] = round(ms, 3)
        print(json.dumps(out), flush=True)
        return
    if args.kernel_only == "nn_forward":
        # the learned stage's forward pass on one nn_ny x nn_nx x 64 grid (256^2: a training crop of
        # 4.2 M voxels; 2048^2: the inference grid of the learned workload)
        from paper_1402_3545_gb300 import learned
        shape = (64, args.nn_ny or args.nn_nx, args.nn_nx)
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
    if args.kernel_only == "panel_smooth":
        # the finest-level Smooth of the cubed-sphere panel operator (512^2 x 128, native FP64)
        pp = workloads.panel()
        pop = tpmg.PanelOperator(pp.nx, pp.ny, pp.nz, pp.omega2, pp.lambda2, pp.H, pp.extent, nlevels=pp.nlevels)
        f = torch.from_numpy(pp.rhs()).cuda().reshape(-1)
        u = torch.zeros_like(f)
        uo = torch.empty_like(f)
        tpmg.panel_smooth(pop.op, pop.L, 2.0 / 3.0, u, f, uo, pp.n)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(max(args.steps, 1)):
            tpmg.panel_smooth(pop.op, pop.L, 2.0 / 3.0, f, f, uo, pp.n)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"kernel": "panel_smooth", "workload": pp.name,
                          "ms_per_launch": round(e0.elapsed_time(e1) / max(args.steps, 1), 4)}), flush=True)
        pop.close()
        return
    p = workloads.mid()
    op = tpmg.Operator.from_problem(p)
    if args.kernel_only == "transpose":
        # host-buffer solves with the vertically contiguous host layout (copies + transposes + solve)
        prm = tpmg.default_params(prec=tpmg.F64, tol=1e-6, max_iter=100, zero_guess=1)
        f_h = torch.from_numpy(np.ascontiguousarray(p.rhs().transpose(1, 2, 0))).reshape(-1).pin_memory()
        u_h = torch.zeros_like(f_h).pin_memory()
        for _ in range(max(args.steps, 1)):
            r = tpmg.mg_solve_host(op.op, prm, f_h, u_h, p.n, layout=tpmg.LAYOUT_Z)
        print(json.dumps({"kernel": "transpose", "workload": p.name, "ms": round(r["ms"], 3),
                          "ms_io": round(r["ms_io"], 3)}), flush=True)
        op.close()
        return
    prec = {"dw": tpmg.DW, "f32": tpmg.F32, "f64": tpmg.F64}[args.precision]
    kid = {"smooth": tpmg.K_SMOOTH, "residual": tpmg.K_RESIDUAL, "restrict_smooth": tpmg.K_RESTRICT_SMOOTH,
           "prolongate": tpmg.K_PROLONGATE, "line_solve": tpmg.K_LINE_SOLVE, "cg_spmv": tpmg.K_CG_SPMV,
           "cg_tridiag": tpmg.K_CG_TRIDIAG, "residual_restrict": tpmg.K_RESIDUAL_RESTRICT,
           "apply_A": tpmg.K_APPLY_A}[args.kernel_only]
    tpmg.op_reserve(op.op, tpmg.MIXED if prec == tpmg.F32 else prec)
    for l in range(1, op.L + 1):
        tpmg.set_variant(op.op, prec, l, args.variant)
    ms = tpmg.time_kernel(op.op, prec, kid, reps=max(args.steps, 1))
    torch.cuda.synchronize()
    print(json.dumps({"kernel": args.kernel_only, "precision": args.precision, "variant": args.variant,
                      "workload": p.name, "ms_per_launch": round(ms, 4)}), flush=True)
    op.close()


def hbm_roofline(tpmg, op, prec, n, peaks, peak_kind, traffic, variant, label, value_bytes):
    """HBM roofline of the finest-level Smooth in precision prec: algorithmic bytes (read u, f; write
    u') over its CUDA-event launch time, against the measured copy rate."""
    t = tpmg.time_kernel(op.op, prec, tpmg.K_SMOOTH, reps=20)
    b = 3 * value_bytes * n
    ach = b / (t * 1e-3) / 1e9
    key = ("smooth", label, int(variant) if variant is not None else -1, "mid_512x512x128")
    tr = traffic.get(key)
    return {"bound": "hbm", "achieved": round(ach, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(ach / peaks["hbm_gbs"], 4), "traffic": tr[0] if tr else None,
            "traffic_source": (f"ncu capture: {tr[1]}" if tr else None),
            "kernel": f"finest-level {label} Smooth (tile variant {variant})", "peak_source": peak_kind,
            "bytes_per_launch": b, "ms_per_launch": round(t, 4)}


def run_ours(args, rank, world, dist):
    import torch
    from paper_1402_3545_gb300 import autotune, tpmg

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = workloads.mid()
    f = p.rhs()
    n = p.n
    op = tpmg.Operator.from_problem(p)
    prec = {"f64": tpmg.F64, "dw": tpmg.DW, "mixed": tpmg.MIXED}[args.solve_precision if args.solve_only else "f64"]
    prm = tpmg.default_params(prec=prec, tol=1e-6, max_iter=100, zero_guess=1)
    tpmg.op_reserve(op.op, prec)
    tuned = {}
    tuned["f64"] = autotune.tune(op, tpmg.F64, lambda_varies=True)
    if prec != tpmg.F64:
        tuned["dw"] = autotune.tune(op, tpmg.DW, lambda_varies=True)
    fd = torch.from_numpy(f).to(dev)
    u = torch.zeros_like(fd)
    stream = torch.cuda.current_stream()

    def solve():  # from u = 0 (zero_guess: the solve clears u itself, u is output only)
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
                              "precision": args.solve_precision, "gpu_launches": int(launches),
                              "solve_only": True}), flush=True)
        op.close()
        return
    sols = {"mid": {"f64": u.cpu().numpy()}}
    sols["mid_headline_u"] = sols["mid"]["f64"]

    # dominant kernel: the finest-level native FP64 Smooth (4 of the 5 fine-level sweeps of each
    # cycle), bound by the FP64 pipe, which issues multiply-adds, adds and multiplies at one rate:
    # FP64 instructions per second over its CUDA-event launch time, against the FP64 instruction
    # rate measured on this GPU in this process (tpmg_measure_alu_rate)
    peaks, peak_kind = measured_peaks()
    traffic = read_traffic()
    fma_rate, _ = tpmg.measure_alu_rate(tpmg.ALU_FP64_FMA)
    add_rate, _ = tpmg.measure_alu_rate(tpmg.ALU_FP64_ADD)
    t_s64 = tpmg.time_kernel(op.op, tpmg.F64, tpmg.K_SMOOTH, reps=20)
    v64 = tuned["f64"][-1] if tuned["f64"] else None
    ach = SMOOTH_F64_INSTR * n / (t_s64 * 1e-3) / 1e12
    peak64 = min(fma_rate, add_rate) / 1e12
    tr = traffic.get(("smooth", "f64", int(v64) if v64 is not None else -1, "mid_512x512x128"))
    roofline = {"bound": "alu", "achieved": round(ach, 4), "peak": round(peak64, 4), "unit": "T FP64 op/s",
                "frac": round(ach / peak64, 4), "traffic": tr[0] if tr else None,
                "traffic_source": (f"ncu capture: {tr[1]}" if tr else None),
                "kernel": f"finest-level native FP64 Smooth (tile variant {v64})",
                "peak_source": ("measured in this run: FP64 instruction rate of tpmg_measure_alu_rate "
                                f"(multiply-add {fma_rate / 1e12:.4f}, add {add_rate / 1e12:.4f} T/s)"),
                "op": "one FP64 arithmetic instruction (multiply-add, add or multiply: the same rate)",
                "ops_per_cell": SMOOTH_F64_INSTR, "ops_per_launch": SMOOTH_F64_INSTR * n,
                "ms_per_launch": round(t_s64, 4),
                "flops": {"per_cell": SMOOTH_F64_FLOPS, "achieved_tflops": round(SMOOTH_F64_FLOPS * n / (t_s64 * 1e-3) / 1e12, 4),
                          "peak_tflops": round(2 * fma_rate / 1e12, 4),
                          "frac": round(SMOOTH_F64_FLOPS * n / (t_s64 * 1e-3) / (2 * fma_rate), 4)},
                "share_of_solve": round((4 * iters[-1] + 1) * t_s64 / ms_per_step, 3),
                "hbm_frac_same_launch": round(3 * 8 * n / (t_s64 * 1e-3) / 1e9 / peaks["hbm_gbs"], 4),
                "hbm_peak_source": peak_kind}
    kernel_ms = {name: round(tpmg.time_kernel(op.op, tpmg.F64, kid, reps=10), 4) for name, kid in [
        ("residual", tpmg.K_RESIDUAL), ("residual_restrict_fused", tpmg.K_RESIDUAL_RESTRICT),
        ("prolongate", tpmg.K_PROLONGATE), ("apply_A", tpmg.K_APPLY_A), ("line_solve", tpmg.K_LINE_SOLVE),
        ("cg_spmv", tpmg.K_CG_SPMV), ("cg_tridiag", tpmg.K_CG_TRIDIAG)]}
    kernel_ms["smooth"] = round(t_s64, 4)

    # the whole solve's useful bandwidth: the paper's per-kernel memory references x 8 B per solve
    level_cells = [0] + [op.level_n(l) for l in range(1, op.L + 1)]
    solve_bytes = 8 * solve_memrefs(level_cells, iters[-1])
    solve_hbm = {"bytes_per_solve": int(solve_bytes), "ms_per_solve": round(value, 4),
                 "achieved": round(solve_bytes / (value * 1e-3) / 1e9, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                 "frac": round(solve_bytes / (value * 1e-3) / 1e9 / peaks["hbm_gbs"], 4), "peak_source": peak_kind,
                 "model": ("memory references of the paper's kernels (Smooth and Residual 3 per cell, "
                           "RestrictSmooth 6 per coarse cell, Prolongate 2.25 per fine cell) x 8 B, "
                           f"{iters[-1]} V(2,2) cycles + the first Smooth")}

    # end to end through the public API with host buffers: tpmg_mg_solve_host on page-locked host
    # fields in the vertically contiguous layout of a CPU code (copy of f to the device, transpose,
    # native FP64 solve, transpose, copy of u back), the paper's "total solution time" (Sec. 5.1)
    f_h = torch.from_numpy(np.ascontiguousarray(f.transpose(1, 2, 0))).reshape(-1).pin_memory()
    u_h = torch.zeros_like(f_h).pin_memory()
    f_hx = torch.from_numpy(f).reshape(-1).pin_memory()
    for _ in range(2):
        tpmg.mg_solve_host(op.op, prm, f_h, u_h, n, layout=tpmg.LAYOUT_Z)
    torch.cuda.synchronize()
    e2e_ms, io_ms = [], []
    for _ in range(args.steps):
        r = tpmg.mg_solve_host(op.op, prm, f_h, u_h, n, layout=tpmg.LAYOUT_Z)
        e2e_ms.append(r["ms"])
        io_ms.append(r["ms_io"])
    rx = [tpmg.mg_solve_host(op.op, prm, f_hx, u_h, n, layout=tpmg.LAYOUT_X)["ms"] for _ in range(2)]
    e2e = {"value": round(float(np.mean(e2e_ms)), 4), "unit": "ms", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n,
           "path": ("tpmg_mg_solve_host, native FP64, page-locked host f and u in the vertically contiguous "
                    "layout: copy + transpose in, solve, transpose + copy out"),
           "copy_and_transpose_ms": round(float(np.mean(io_ms)), 4),
           "x_layout_ms": round(min(rx), 4)}

    # the other precisions and CG on the same problem (after a warm-up solve each); DW and the
    # mixed solver's FP32 Smooth get their own HBM rooflines
    variants = {}
    tuned.setdefault("dw", autotune.tune(op, tpmg.DW, lambda_varies=True))
    tpmg.op_reserve(op.op, tpmg.MIXED)
    tuned["f32"] = autotune.tune(op, tpmg.F32, lambda_varies=True)
    for name, vprec, tol, bf in [("dw", tpmg.DW, 1e-6, 0), ("mixed", tpmg.MIXED, 1e-6, 0),
                                 ("mixed_1e-10", tpmg.MIXED, 1e-10, 0), ("mixed_bf16_coarse", tpmg.MIXED, 1e-6, 1)]:
        vp = tpmg.default_params(prec=vprec, tol=tol, max_iter=100, coarse_bf16=bf, zero_guess=1)
        ms = []
        for _ in range(3):
            r = tpmg.mg_solve(op.op, vp, fd, u, n)
            ms.append(r["ms"])
        variants[name] = {"ms": round(min(ms[1:]), 3), "iters": r["iters"], "rel_res": r["rel_res"],
                          "speedup_vs_f64": round(value / min(ms[1:]), 3)}
        if not bf:
            sols["mid"][name] = u.cpu().numpy()
    variants["dw"]["roofline"] = hbm_roofline(tpmg, op, tpmg.DW, n, peaks, peak_kind, traffic, tuned["dw"][-1],
                                              "dw", 8)
    variants["mixed"]["roofline_f32_smooth"] = hbm_roofline(tpmg, op, tpmg.F32, n, peaks, peak_kind, traffic,
                                                            tuned["f32"][-1], "f32", 4)
    variants["dw"]["kernel_ms"] = {name: round(tpmg.time_kernel(op.op, tpmg.DW, kid, reps=10), 4) for name, kid in [
        ("smooth", tpmg.K_SMOOTH), ("residual", tpmg.K_RESIDUAL), ("residual_restrict_fused", tpmg.K_RESIDUAL_RESTRICT),
        ("prolongate", tpmg.K_PROLONGATE), ("apply_A", tpmg.K_APPLY_A), ("cg_spmv", tpmg.K_CG_SPMV),
        ("cg_tridiag", tpmg.K_CG_TRIDIAG)]}
    variants["mixed"]["kernel_ms_f32"] = {name: round(tpmg.time_kernel(op.op, tpmg.F32, kid, reps=10), 4)
                                          for name, kid in [
        ("smooth", tpmg.K_SMOOTH), ("residual", tpmg.K_RESIDUAL), ("line_solve", tpmg.K_LINE_SOLVE),
        ("residual_restrict_fused", tpmg.K_RESIDUAL_RESTRICT), ("prolongate", tpmg.K_PROLONGATE)]}
    for name, vprec in [("cg_f64", tpmg.F64), ("cg_dw", tpmg.DW)]:
        r = tpmg.cg_solve(op.op, tpmg.default_params(prec=vprec, tol=1e-6, max_iter=5000, zero_guess=1), fd, u, n)
        variants[name] = {"ms": round(r["ms"], 3), "iters": r["iters"], "rel_res": r["rel_res"]}
        sols["mid"][name] = u.cpu().numpy()
    variants["batched_64"] = bench_batched(tpmg, torch, sols)
    variants["mixed_1024x1024x128"] = bench_mixed(tpmg, torch, sols)
    variants["paper_shaped_512x512x128"] = bench_paper_shaped(tpmg, torch)
    variants["robustness_512x512x128"] = bench_robustness(tpmg, torch)
    variants["panel_512x512x128"] = bench_panel(tpmg, torch, sols)
    variants["learned_2048x2048x64"] = bench_learned(tpmg, torch, sols)

    cpu, errors = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, errors = cpu_leg(p, f, sols)
    del sols

    if rank == 0:
        line = {"metric": METRIC, "value": round(value, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4), "higher_is_better": False,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": p.name, "nx": p.nx, "ny": p.ny, "nz": p.nz, "levels": op.L,
                           "solver": "V(2,2), rho 0.8, 2 coarse steps", "tol": 1e-6,
                           "precision": "native FP64", "parallelism": f"replicas{world}",
                           "l2": "inputs larger than L2 (268 MB per FP64 field > 129 MB)"},
                "iters": iters[-1], "roofline": roofline, "solve_hbm": solve_hbm, "kernel_ms": kernel_ms,
                "tile_variants": tuned, "variants": variants, "errors_vs_reference": errors,
                "e2e": e2e, "cpu_baseline": cpu, "clocks": clocks, "gpu_launches": int(launches)}
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
