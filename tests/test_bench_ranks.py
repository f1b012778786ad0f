"""The multi-rank logic of bench.py on CPU, with world_size-2 gloo ranks.

Under torchrun every rank solves its own copy of the instance (replicas, no
data-path collective).  The timing is reduced to the slowest rank, and the
whole-job value counts every rank's ant-solutions over that time.  The
reference arm runs on rank 0 alone.
"""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, ms_of_rank, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(ms_of_rank[rank], world, "cpu")
        out[rank] = (ms, bench.job_throughput(1024 * 100, world, ms))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    world, port = 2, free_port()
    ms_of_rank = [1500.0, 1750.0]
    out = mp.Manager().dict()
    mp.spawn(rank_main, args=(world, port, ms_of_rank, out), nprocs=world, join=True)
    for rank in range(world):
        ms, value = out[rank]
        assert ms == 1750.0
        assert value == pytest.approx(2 * 1024 * 100 / 1.75)


def test_one_rank_needs_no_collective():
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.job_throughput(1024 * 100, 1, 2000.0) == pytest.approx(51200.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")

    class Args:
        workload = "stippled100k"
        warmup = 3
        steps = 3
        ref_ants = 32
        gpus = 2

    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(Args(), {"ants": 1024, "iters": 100, "n": 100_000})
    assert buf.getvalue() == ""
