"""The multi-GPU path of the benchmark is replicas only (one independent solve per rank, no
collective on the data path); its timing aggregation -- the slowest rank's time, every rank solving
its own copies -- and the reference arm's rank-0-only rule, checked with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [120.0, 150.0][rank]  # rank 1 is the slow one
        m = bench.max_over_ranks(elapsed, dist, torch.device("cpu"))
        out[rank] = (m, bench.per_solve_ms(m, steps=5, world=world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    world = 2
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        m, v = out[r]
        assert m == 150.0
        assert v == pytest.approx(150.0 / (5 * world))


def test_single_process_needs_no_collective():
    assert bench.max_over_ranks(3.5, None, None) == 3.5
    assert bench.per_solve_ms(100.0, 4, 1) == 25.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        steps, warmup = 1, 0

    # rank 1 of 2 returns at once without touching the oracle or printing a line
    assert bench.run_reference(Args(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""
