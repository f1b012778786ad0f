#!/usr/bin/env python3
"""Benchmark: Focused ACO on the n = 100,000 stippled workload (1,024 ants,
100 iterations, k = 16, Philox seed 1) on GB300.

One step = one full solve of that instance through the library: colony
set-up from device-resident coordinates (candidate/backup lists, initial
tour), 100 iterations of 1,024 ants (focused construction + local search +
colony update), and the global-best tour copied to a device buffer.

  value     ant-solutions per second of the whole job (ants * iterations *
            ranks / step time), CUDA events on the colony's stream;
  e2e       the same metric through the public host API (faco_create_ex from
            pinned host coordinates, faco_iterate, faco_best into a host
            array), host<->device copies inside the timed region;
  roofline  the per-ant kernel (construction + local search), timed live
            with CUDA events around each launch; achieved = algorithmic
            bytes / kernel time against the measured HBM copy bandwidth;
  cpu_baseline  the CPU oracle on a bounded sample of the same workload.

L2 is flushed (a 512 MB write) before every timed step.  Under torchrun each
rank solves its own copy of the instance (independent colonies, no data-path
collective): weak scaling.

Two more sections ride on the same line (both on by default, --sections):
  batched   512 independent instances (n log-uniform in [200, 20,000], 64
            ants, 100 iterations) as one Batch -- one graph launch for the
            budget -- vs. the plain one-Colony-at-a-time loop on a
            stratified sample of the same instances (instances/s);
  served    a Poisson stream of requests (n log-uniform in [1,000,
            100,000], 256 ants, 50 iterations) through the Server vs. the
            plain loop on the same trace (p50/p99 time-to-budget,
            instances/s).
Each carries its own oracle timing on a bounded sample.

--impl reference times the CPU oracle instead (the method's plain
statement, test infrastructure) on a bounded sample of the same workload.
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

METRIC = "ant-solutions/sec at 100k nodes"
UNIT = "ant-solutions/s"


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest of the ranks' values, on every rank (x itself on one
    rank).  `device` holds the reduced tensor: the GPU under NCCL, "cpu"
    under gloo."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms: float) -> float:
    """Whole-job throughput: the units of every rank over the slowest
    rank's time (ms)."""
    return units_per_rank * world / (ms / 1e3)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for name, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def host_cores() -> int:
    return os.cpu_count() or 1


# Sources of the per-ant kernel; the DRAM traffic recorded under profiles/
# applies only while their hash matches the one recorded with it.
ANTS_SOURCES = ["ants.cuh", "ants_blk_body.inc", "ls.cuh", "seg.cuh", "nearest.cuh", "common.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "k_ants_blk_stippled100k_traffic.json")


def ants_sources_hash() -> str:
    import hashlib

    h = hashlib.sha256()
    for f in ANTS_SOURCES:
        with open(os.path.join(ROOT, "paper_2203_02228_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def recorded_traffic():
    """DRAM bytes per launch of the per-ant kernel from one ncu capture, or
    None when the kernel changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
        if rec.get("sources_sha256") == ants_sources_hash():
            return float(rec["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


def oracle_sample(xy, ants, iters, k, sample_ants, sample_iters, threads):
    """Times the oracle's set-up and `sample_iters` iterations of
    `sample_ants` ants; returns the full-job throughput implied by them."""
    import oracle

    t0 = time.perf_counter()
    col = oracle.Colony(xy, k, threads=threads)
    t_create = time.perf_counter() - t0
    t0 = time.perf_counter()
    col.iterate(sample_ants, sample_iters)
    t_iter = (time.perf_counter() - t0) / (sample_iters * sample_ants)  # seconds per ant-solution
    col.close()
    t_job = t_create + t_iter * ants * iters
    return ants * iters / t_job, t_create, t_iter


def run_reference(args, W):
    """The CPU oracle as the reference arm (rank 0 only)."""
    from paper_2203_02228_gb300 import inputs

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    xy = inputs.workload_points(args.workload)
    threads = host_cores()
    vals = []
    for s in range(args.warmup + args.steps):
        v, tc, ti = oracle_sample(xy, W["ants"], W["iters"], 16, args.ref_ants, 1, threads)
        if s >= args.warmup:
            vals.append(v)
    v = statistics.mean(vals)
    sample = ("per step: oracle set-up of the full instance + 1 iteration of %d ants; value = "
              "ants*iterations / (set-up + per-ant time * %d ants * %d iterations)") % (
        args.ref_ants, W["ants"], W["iters"])
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": W["ants"] * W["iters"] / v * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+int64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": W["n"], "ants": W["ants"], "iterations": W["iters"],
                   "k": 16, "seed": 1},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def bench_batched(args, stream, flush, barrier):
    """The 512-instance batch (one Batch: set-up of every instance, 64 ants x
    100 iterations in one graph launch, every tour back to the host) against
    the plain one-instance-at-a-time loop (Colony per instance through the
    same host API) on a stratified sample of the same instances."""
    import torch

    from paper_2203_02228_gb300 import Batch, Colony, inputs

    w = inputs.BATCH_WORKLOADS["batch512"]
    xs, seeds = inputs.batch_workload("batch512")
    ants, iters, k = w["ants"], w["iters"], w["k"]
    ns = np.array([x.shape[0] for x in xs])
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def run_batch():
        b = Batch(xs, k, seeds=seeds, stream=stream)
        b.iterate(ants, iters)
        tours, lens = b.tours()
        return b, tours, lens

    for _ in range(2):  # the first also runs the kernel tuner (cached per process)
        b, _, _ = run_batch()
        b.close()
    times, wall = [], []
    for _ in range(max(1, args.batch_steps)):
        flush.zero_()
        barrier()
        e0, e1 = ev(), ev()
        t0 = time.perf_counter()
        e0.record(stream)
        b, tours, lens = run_batch()
        e1.record(stream)
        e1.synchronize()
        wall.append(time.perf_counter() - t0)
        times.append(e0.elapsed_time(e1) / 1e3)
        plan = b.plan()
        launches = b.stats(0).kernel_launches
        b.close()
    t_batch = statistics.mean(wall)

    # plain loop on every 8th instance by size: the sample spans the size range
    order = np.argsort(ns, kind="stable")
    sample = order[4::8]
    Colony(xs[int(sample[0])], k, seed=int(seeds[sample[0]])).close()  # warm
    flush.zero_()
    barrier()
    t0 = time.perf_counter()
    plain = {}
    for i in sample:
        c = Colony(xs[int(i)], k, seed=int(seeds[i]), stream=stream)
        c.iterate(ants, iters)
        plain[int(i)] = c.best()
        c.close()
    t_plain = time.perf_counter() - t0
    same = all(np.array_equal(plain[i][0], tours[i]) and plain[i][1] == lens[i] for i in plain)
    inst_batch = len(xs) / t_batch
    inst_plain = len(sample) / t_plain
    cpu = None
    if not args.no_cpu:
        # the oracle on 8 instances spread over the sizes: set-up + 1 iteration
        # of the 64 ants, extrapolated to 100 iterations; instances/s of the
        # whole batch = 512 / (64 x the sample's time)
        import oracle

        osample = order[32::64]
        t_sum = 0.0
        for i in osample:
            t0 = time.perf_counter()
            col = oracle.Colony(xs[int(i)], k, seed=int(seeds[i]), threads=host_cores())
            t1 = time.perf_counter()
            col.iterate(ants, 1)
            t2 = time.perf_counter()
            col.close()
            t_sum += (t1 - t0) + iters * (t2 - t1)
        cpu = {"value": len(osample) / t_sum, "unit": "instances/s", "cores": host_cores(), "kind": "oracle",
               "sample": "%d of %d instances (every 64th by size): oracle set-up + 1 iteration of %d ants, "
                         "extrapolated to %d iterations" % (len(osample), len(xs), ants, iters)}
    return {
        "workload": "batch512", "instances": len(xs), "n_range": [int(ns.min()), int(ns.max())],
        "n_mean": float(ns.mean()), "ants": ants, "iterations": iters, "k": k,
        "metric": "instances/sec (set-up + budget + tours to host)", "unit": "instances/s",
        "value": inst_batch, "ms_per_batch": t_batch * 1e3, "device_ms_per_batch": statistics.mean(times) * 1e3,
        "ant_solutions_per_s": len(xs) * ants * iters / t_batch,
        "plain_loop": {"value": inst_plain, "unit": "instances/s", "sample": "%d of %d instances (every 8th by "
                       "size), one Colony each through the same host API" % (len(sample), len(xs)),
                       "seconds": t_plain},
        "speedup_vs_plain": inst_batch / inst_plain,
        "equal_results_on_sample": bool(same),
        "mean_best_length": float(np.mean(lens)),
        "plan": {"colonies_per_kernel": {name: int((plan == v).sum()) for v, name in
                                         enumerate(("segment_table", "arrays_2_blocks_per_sm", "arrays_4_blocks_per_sm",
                                                    "arrays_8_blocks_per_sm"))}},
        "gpu_launches_per_batch": int(launches), "graph_launches_per_batch": 1, "cpu_baseline": cpu,
        "h2d_bytes_per_batch": int(8 * ns.sum()), "d2h_bytes_per_batch": int(4 * ns.sum() + 8 * len(xs)),
    }


def bench_served(args, stream, barrier):
    """A Poisson stream of requests (n log-uniform in [1e3, 1e5], 256 ants,
    50 iterations) through the server -- admission by device memory,
    continuous batching -- and the same arrival trace through the plain
    loop (one Colony at a time, first come first served).  Time-to-budget
    = completion - arrival, host clock."""
    import threading as th

    from paper_2203_02228_gb300 import Colony, Server, inputs

    w = inputs.SERVE_WORKLOADS["serve100k"]
    out = {"workload": "serve100k", "ants": w["ants"], "iterations": w["iters"], "k": w["k"],
           "n_range": [w["lo"], w["hi"]], "metric": "time-to-budget p50/p99 (s), instances/sec",
           "pool_bytes": args.serve_pool_gb << 30, "rates": []}
    # warm: kernel tuner and module load, outside the timed streams
    with Server(1 << 30) as s:
        for j, n in enumerate((1500, 6000, 30000)):
            s.wait(s.submit(inputs.uniform(n, seed=j), w["k"], w["ants"], 2, 1))
    for rate in args.serve_rates:
        xs, seeds, arr = inputs.serve_trace("serve100k", args.serve_requests, rate)
        # served
        barrier()
        with Server(args.serve_pool_gb << 30) as s:
            t0 = time.perf_counter()
            tickets = [None] * len(xs)

            def feed():
                for i, x in enumerate(xs):
                    d = t0 + arr[i] - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    tickets[i] = s.submit(x, w["k"], w["ants"], w["iters"], int(seeds[i]))

            f = th.Thread(target=feed)
            f.start()
            f.join()
            res = [s.wait(t) for t in tickets]
            st = s.stats()
        lat = np.array([(r[3] - r[2]) / 1e9 for r in res])
        span = (max(r[3] for r in res) - min(r[2] for r in res)) / 1e9
        served = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                  "mean_s": float(lat.mean()), "instances_per_s": len(xs) / span,
                  "ant_solutions_per_s": len(xs) * w["ants"] * w["iters"] / span,
                  "peak_active": st["peak_active"], "rounds": st["rounds"],
                  "gpu_launches": st["kernel_launches"], "mean_best_length": float(np.mean([r[1] for r in res]))}
        # plain loop, same trace: one instance at a time in arrival order
        barrier()
        t0 = time.perf_counter()
        plat, plens = [], []
        for i, x in enumerate(xs):
            d = t0 + arr[i] - time.perf_counter()
            if d > 0:
                time.sleep(d)
            c = Colony(x, w["k"], seed=int(seeds[i]), stream=stream)
            c.iterate(w["ants"], w["iters"])
            tour, L = c.best()
            c.close()
            plat.append(time.perf_counter() - (t0 + arr[i]))
            plens.append(L)
        pspan = time.perf_counter() - t0
        plat = np.array(plat)
        plain = {"p50_s": float(np.percentile(plat, 50)), "p99_s": float(np.percentile(plat, 99)),
                 "mean_s": float(plat.mean()), "instances_per_s": len(xs) / pspan}
        out["rates"].append({"rate_per_s": rate, "requests": len(xs), "served": served, "plain_loop": plain,
                             "equal_lengths": bool(np.array_equal([r[1] for r in res], plens))})
    if not args.no_cpu:
        # the oracle on three requests of the trace (10th, 50th, 90th size
        # percentile): set-up + 1 iteration of 32 ants, scaled to 256 ants x 50
        import oracle

        xs, seeds, _ = inputs.serve_trace("serve100k", args.serve_requests, args.serve_rates[0])
        ns = np.array([x.shape[0] for x in xs])
        order = np.argsort(ns)
        pick = [order[int(q * (len(xs) - 1))] for q in (0.1, 0.5, 0.9)]
        t_sum = 0.0
        for i in pick:
            t0 = time.perf_counter()
            col = oracle.Colony(xs[int(i)], w["k"], seed=int(seeds[i]), threads=host_cores())
            t1 = time.perf_counter()
            col.iterate(32, 1)
            t2 = time.perf_counter()
            col.close()
            t_sum += (t1 - t0) + w["iters"] * (t2 - t1) * w["ants"] / 32
        out["cpu_baseline"] = {"value": len(pick) / t_sum, "unit": "instances/s", "cores": host_cores(),
                               "kind": "oracle", "sample": "3 requests (10th/50th/90th size percentile, n = %s): "
                               "oracle set-up + 1 iteration of 32 ants, scaled to %d ants x %d iterations; one "
                               "request at a time" % ([int(ns[i]) for i in pick], w["ants"], w["iters"])}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="faco", choices=["faco", "reference"])
    ap.add_argument("--workload", default="stippled100k")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--ref-ants", type=int, default=32)
    ap.add_argument("--iters", type=int, default=0, help="override the iteration budget (testing only)")
    ap.add_argument("--sections", default="main,batch,serve", help="comma list of: main, batch, serve")
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[2.0, 8.0])
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-pool-gb", type=int, default=64)
    args = ap.parse_args()
    sections = set(args.sections.split(","))

    from paper_2203_02228_gb300 import inputs

    W = dict(inputs.WORKLOADS[args.workload])
    if args.iters:
        W["iters"] = args.iters
    if args.impl == "reference":
        return run_reference(args, W)

    import torch
    import torch.distributed as dist

    from paper_2203_02228_gb300 import Colony, build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)

    xy = inputs.workload_points(args.workload)
    n, ants, iters = xy.shape[0], W["ants"], W["iters"]
    xy_dev = torch.from_numpy(xy).to(dev)
    tour_dev = torch.empty(n, dtype=torch.int32, device=dev)
    len_dev = torch.empty(1, dtype=torch.int64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def solve(profile=False):
        col = Colony(xy_dev, 16, device=True, stream=stream)
        if profile:
            col.profile(True)
        col.iterate(ants, iters)
        col.best_device(tour_dev, len_dev)
        st = col.stats()
        prof = col.profile_read() if profile else (0.0, 0)
        col.close()
        return st, prof

    if "main" not in sections:
        out = {}
        if "batch" in sections:
            out["batched"] = bench_batched(args, stream, flush, barrier)
        if "serve" in sections:
            out["served"] = bench_served(args, stream, barrier)
        if rank == 0:
            print(json.dumps(out), flush=True)
        return

    for _ in range(args.warmup):
        solve()
    barrier()

    clocks = ClockSampler(local)
    clocks.start()
    step_ms = []
    ants_ms = 0.0
    ants_launches = 0
    algo_bytes = 0
    launches = 0
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, (pms, pcnt) = solve(profile=True)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        ants_ms += pms
        ants_launches += pcnt
        launches += st.kernel_launches
        # algorithmic bytes of the per-ant kernel: explicit route+pos per ant
        # (16n), source rows per roulette step (2 x 64 B + visited/route 16 B),
        # 16 B per reversed element, 2k x 20 B per local-search pop.
        algo_bytes += (16 * n * ants * iters + 208 * st.aco_steps + 16 * st.flip_elems + 640 * st.ls_pops)
    barrier()
    clk = clocks.stop()

    ms = max_over_ranks(statistics.mean(step_ms), world, dev)
    value = job_throughput(ants * iters, world, ms)

    # end to end through the host API (pinned host coordinates, host tour)
    e2e = None
    if not args.no_e2e:
        from paper_2203_02228_gb300 import _lib, faco_best, faco_create_ex, faco_destroy, faco_iterate
        pinned = torch.from_numpy(xy).pin_memory()
        tour_host = np.zeros(n, np.int32)
        p = _lib.params_default()
        p.stream = stream.cuda_stream
        e2e_ms = []
        for _ in range(max(1, args.steps)):
            flush.zero_()
            barrier()
            t0 = time.perf_counter()
            h = faco_create_ex(pinned, n, 16, p)
            faco_iterate(h, ants, iters)
            faco_best(h, tour_host, n)
            t1 = time.perf_counter()
            faco_destroy(h)
            e2e_ms.append((t1 - t0) * 1e3)
        em = max_over_ranks(statistics.mean(e2e_ms), world, dev)
        e2e = {"value": job_throughput(ants * iters, world, em), "unit": UNIT, "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": 4 * n + 8, "ms_per_step": em}

    peak, peak_src = load_peaks()
    achieved = (algo_bytes / ants_launches) / (ants_ms / ants_launches / 1e3) / 1e9 if ants_launches else None
    roofline = {"kernel": "k_ants_blk (construction + local search)", "bound": "hbm", "achieved": achieved,
                "peak": peak, "peak_source": peak_src, "unit": "GB/s",
                "frac": achieved / peak if achieved else None, "traffic": recorded_traffic(),
                "avg_launch_ms": ants_ms / ants_launches if ants_launches else None,
                "algorithmic_bytes_per_launch": algo_bytes / ants_launches if ants_launches else None}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, tc, ti = oracle_sample(xy, ants, iters, 16, 32, 1, host_cores())
        cpu = {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": "oracle set-up of the full instance (%.1f s) + 1 iteration of 32 ants (%.1f ms per "
                         "ant-solution), extrapolated to %d ants x %d iterations" % (tc, ti * 1e3, ants, iters)}

    batched = served = None
    if "batch" in sections and world == 1:
        batched = bench_batched(args, stream, flush, barrier)
    if "serve" in sections and world == 1:
        served = bench_served(args, stream, barrier)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+int64", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "ants": ants, "iterations": iters, "k": 16,
                       "seed": 1, "l2": "flushed before every step (512 MB write)",
                       "parallelism": "independent colonies per rank" if world > 1 else "single colony"},
            "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk, "batched": batched, "served": served,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
