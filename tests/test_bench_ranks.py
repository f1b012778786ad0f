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


def test_plain_loop_times_follow_first_come_first_served():
    """The plain loop serves one request at a time in arrival order:
    completion C_i = max(A_i, C_{i-1}) + S_i (checked by an explicit event
    simulation of a single server)."""
    import numpy as np

    rng = np.random.default_rng(3)
    for _ in range(20):
        m = int(rng.integers(1, 40))
        arr = np.cumsum(rng.exponential(0.3, m))
        svc = rng.uniform(0.05, 0.8, m)
        got = bench.plain_loop_times(arr, svc)
        t, busy_until = 0.0, 0.0
        want = []
        for a_i, s_i in zip(arr, svc):  # the server idles until the next arrival
            t = a_i if a_i > busy_until else busy_until
            busy_until = t + s_i
            want.append(busy_until)
        np.testing.assert_allclose(got, want)
        assert np.all(got - arr >= svc - 1e-12)


def test_serve_plan_caps_the_lowest_rates():
    plan = dict(bench.serve_plan([1, 2, 5, 10, 200], 100))
    assert plan[1] == 30 and plan[2] == 60 and plan[5] == 100 and plan[10] == 100 and plan[200] == 100
    assert dict(bench.serve_plan([0.5], 100))[0.5] == 30


def test_roofline_line_rates():
    r = bench.roofline_line("k", 100, 4, 10, ants_ms=20.0, ants_launches=10, algo_bytes=10 * 6e9, peak=6000.0,
                            peak_src="measured", l2_peak=12000.0, traffic=(1e8, 5e9))
    assert abs(r["avg_launch_ms"] - 2.0) < 1e-12
    assert abs(r["achieved"] - 3000.0) < 1e-9 and abs(r["frac"] - 0.5) < 1e-12
    assert abs(r["dram_gbs"] - 50.0) < 1e-9 and abs(r["l2_gbs"] - 2500.0) < 1e-9
    assert abs(r["l2_frac"] - 2500.0 / 12000.0) < 1e-12
    assert bench.roofline_line("k", 1, 1, 1, 0.0, 0, 0, 1.0, "m", None) is None
