"""Host logic of a multi-process bench run, on CPU with the gloo backend
(world size 2): the job's step time is the slowest rank's, the job's
throughput counts the points of every rank, and under torchrun only rank 0
runs the oracle arm."""
import os
import socket
import sys
from pathlib import Path

import torch.multiprocessing as mp

ROOT = Path(__file__).resolve().parents[1]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, str(ROOT))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(100.0 + 25.0 * rank, dist, "cpu")
        q.put((rank, ms, bench.job_throughput(40000, world, ms)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_step_time_is_max_over_ranks_and_throughput_counts_all_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in got:
        assert ms == 125.0, rank
        assert abs(value - 2 * 40000 / 0.125) < 1e-6, rank


def test_single_process_needs_no_process_group():
    sys.path.insert(0, str(ROOT))
    import bench

    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_throughput(40000, 1, 1000.0) == 40000.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, str(ROOT))
    import argparse

    import bench

    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.run_reference(args, 1, 2) is None
    assert capsys.readouterr().out == ""
