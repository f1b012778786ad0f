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
            with CUDA events around each launch: achieved = algorithmic
            bytes / kernel time against the measured HBM copy bandwidth,
            beside the DRAM and L2 rates of the recorded ncu counters (L2
            against the L2 read bandwidth probed in the same run);
  cpu_baseline  the CPU oracle on a bounded sample of the same workload:
            its set-up in full, a few warm-up iterations, then one measured
            iteration on all host cores and one on a single thread.

L2 is flushed (a 512 MB write) before every timed step.  Under torchrun each
rank solves its own copy of the instance (independent colonies, no data-path
collective): weak scaling.

More sections ride on the same line (all on by default, --sections):
  uniform1k     the n = 1,000 workload (32 ants, 200 iterations) in full on
                the GPU, and the oracle's full run on one and on all cores;
  stippled200k  the n = 200,000 workload (256 blobs, 2,048 ants, 50
                iterations): throughput, roofline and an oracle sample;
  batched   512 independent instances (n log-uniform in [200, 20,000], 64
            ants, 100 iterations) as one Batch -- one graph launch for the
            budget -- vs. the plain one-Colony-at-a-time loop on a
            stratified sample of the same instances (instances/s), the
            tuner's per-class timings and the all-segment-table plan;
  served    a Poisson stream of requests (n log-uniform in [1,000,
            100,000], 256 ants, 50 iterations) through the Server at rates
            1..200 per second vs. the plain loop on the same trace (p50/p99
            time-to-budget, instances/s).

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
    """ncu counters of one launch of the per-ant kernel on the n = 100,000
    workload (DRAM bytes, L2 bytes), or None when the kernel changed since."""
    try:
        with open(TRAFFIC_FILE) as f:
            rec = json.load(f)
        if rec.get("sources_sha256") == ants_sources_hash():
            return float(rec["dram_bytes_per_launch"]), float(rec["lts_bytes_per_launch"])
    except Exception:
        pass
    return None


def oracle_steady(xy, k, threads, warm_ants=32, warm_iters=8, sample_all=256, sample_single=16, seed=1):
    """Times the oracle on one instance: its set-up in full (all cores),
    `warm_iters` untimed iterations of `warm_ants` ants (the source moves
    off the initial tour, as in the steady state), then one iteration of
    `sample_all` ants on all cores and one of `sample_single` ants on one
    thread.  Returns (set-up s, s per ant-solution all cores, s per
    ant-solution single thread)."""
    import oracle

    t0 = time.perf_counter()
    col = oracle.Colony(xy, k, threads=threads, seed=seed)
    t_setup = time.perf_counter() - t0
    if warm_iters:
        col.iterate(warm_ants, warm_iters)
    t0 = time.perf_counter()
    col.iterate(sample_all, 1)
    t_all = (time.perf_counter() - t0) / sample_all
    col.set_threads(1)
    t0 = time.perf_counter()
    col.iterate(sample_single, 1)
    t_one = (time.perf_counter() - t0) / sample_single
    col.close()
    return t_setup, t_all, t_one


def cpu_baseline_line(xy, ants, iters, k, threads, **kw):
    """cpu_baseline object: the oracle's whole-job throughput on all cores,
    estimated from its measured set-up and a measured steady iteration
    sample (labelled as such), with the single-thread rate beside it."""
    t_setup, t_all, t_one = oracle_steady(xy, k, threads, **kw)
    sa, so = kw.get("sample_all", 256), kw.get("sample_single", 16)
    v = ants * iters / (t_setup + ants * iters * t_all)
    return {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "extrapolated": True,
            "sample": "oracle set-up of the full instance measured (%.2f s, %d threads); after %d warm-up "
                      "iterations of %d ants, one iteration of %d ants measured on all cores (%.3f ms per "
                      "ant-solution) and one of %d ants on one thread (%.3f ms); value = %d ants x %d "
                      "iterations / (set-up + that many ant-solutions at the all-core rate)" % (
                          t_setup, threads, kw.get("warm_iters", 8), kw.get("warm_ants", 32), sa,
                          t_all * 1e3, so, t_one * 1e3, ants, iters),
            "setup_s": t_setup,
            "all_cores": {"ant_solutions_per_s": 1.0 / t_all, "cores": threads, "sample_ants": sa},
            "single_thread": {"ant_solutions_per_s": 1.0 / t_one, "cores": 1, "sample_ants": so,
                              "note": "iterations only, set-up excluded"}}


def run_reference(args, W):
    """The CPU oracle as the reference arm (rank 0 only): its set-up of the
    full instance and a few warm-up iterations first (untimed), then each
    step is one iteration of --ref-ants ants on all host cores, timed; value
    = ant-solutions per second of those iterations (set-up excluded, which
    favours the oracle against the GPU line, whose steps include set-up)."""
    from paper_2203_02228_gb300 import inputs

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    xy = inputs.workload_points(args.workload)
    threads = host_cores()
    ref_ants = getattr(args, "ref_ants", 128)
    warm_iters = getattr(args, "ref_warm_iters", 8)
    t0 = time.perf_counter()
    col = oracle.Colony(xy, 16, threads=threads)
    t_setup = time.perf_counter() - t0
    col.iterate(32, warm_iters)
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        col.iterate(ref_ants, 1)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    col.close()
    t_step = statistics.mean(times)
    v = ref_ants / t_step
    full = W["ants"] * W["iters"] / (t_setup + W["ants"] * W["iters"] * t_step / ref_ants)
    sample = ("set-up of the full instance (%.2f s) and %d warm-up iterations of 32 ants untimed; each step = one "
              "iteration of %d ants on %d threads, measured; value = ant-solutions/s of the steps (set-up "
              "excluded)" % (t_setup, warm_iters, ref_ants, threads))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+int64",
        "data": "synthetic",
        "config": {"workload": args.workload, "n": W["n"], "ants": W["ants"], "iterations": W["iters"],
                   "k": 16, "seed": 1, "step": "one iteration of %d ants" % ref_ants},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample,
                         "setup_s": t_setup, "full_job_estimate": full},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def roofline_line(kernel, n, ants, iters, ants_ms, ants_launches, algo_bytes, peak, peak_src, l2_peak,
                  traffic=None):
    """The per-ant kernel's roofline object (see the module docstring)."""
    if not ants_launches:
        return None
    t = ants_ms / ants_launches / 1e3  # s per launch
    achieved = algo_bytes / ants_launches / t / 1e9
    r = {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": peak,
         "peak_source": "%s HBM copy bandwidth" % peak_src, "unit": "GB/s", "frac": achieved / peak,
         "achieved_kind": "algorithmic bytes per launch (explicit route/pos arrays per ant, the paper's "
                          "representation) / live CUDA-event launch time",
         "traffic": traffic[0] if traffic else None, "avg_launch_ms": t * 1e3,
         "algorithmic_bytes_per_launch": algo_bytes / ants_launches, "l2_peak": l2_peak,
         "l2_peak_source": "faco_l2_probe in this run (48 MiB resident, 16-byte L1-bypassing reads)"}
    if traffic:
        r["dram_gbs"] = traffic[0] / t / 1e9
        r["dram_frac"] = r["dram_gbs"] / peak
        r["l2_bytes_per_launch"] = traffic[1]
        r["l2_gbs"] = traffic[1] / t / 1e9
        r["l2_frac"] = r["l2_gbs"] / l2_peak if l2_peak else None
    return r


def algorithmic_bytes(n, ants, iters, st):
    """Bytes the paper's explicit-array construction + local search must
    move: route+pos per ant (16n), two 64-byte candidate rows plus 16 bytes
    of visited/route per roulette step, 16 B per reversed element, 2k x 20 B
    per local-search pop."""
    return 16 * n * ants * iters + 208 * st.aco_steps + 16 * st.flip_elems + 640 * st.ls_pops


def bench_colony(xy, ants, iters, steps, warmup, stream, flush, barrier, dev):
    """Full solves of one instance (set-up from device coordinates +
    budget + best tour to a device buffer): step times, per-ant kernel
    time and launches, algorithmic bytes and launch counts of the timed
    steps."""
    import torch

    from paper_2203_02228_gb300 import Colony

    n = xy.shape[0]
    xy_dev = torch.from_numpy(xy).to(dev)
    tour_dev = torch.empty(n, dtype=torch.int32, device=dev)
    len_dev = torch.empty(1, dtype=torch.int64, device=dev)

    def solve(profile):
        col = Colony(xy_dev, 16, device=True, stream=stream)
        if profile:
            col.profile(True)
        col.iterate(ants, iters)
        col.best_device(tour_dev, len_dev)
        st = col.stats()
        prof = col.profile_read() if profile else (0.0, 0)
        col.close()
        return st, prof

    for _ in range(warmup):
        solve(False)
    barrier()
    out = {"step_ms": [], "ants_ms": 0.0, "ants_launches": 0, "algo_bytes": 0, "launches": 0}
    for _ in range(steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, (pms, pcnt) = solve(True)
        e1.record(stream)
        e1.synchronize()
        out["step_ms"].append(e0.elapsed_time(e1))
        out["ants_ms"] += pms
        out["ants_launches"] += pcnt
        out["launches"] += st.kernel_launches
        out["algo_bytes"] += algorithmic_bytes(n, ants, iters, st)
        out["best_length"] = int(len_dev.item())
    return out


def bench_uniform1k(args, stream, flush, barrier, dev):
    """The n = 1,000 workload in full: the GPU (set-up + 32 ants x 200
    iterations, CUDA events) and the oracle's full run, measured, on one
    thread and on all host cores."""
    from paper_2203_02228_gb300 import inputs

    W = inputs.WORKLOADS["uniform1k"]
    xy = inputs.workload_points("uniform1k")
    r = bench_colony(xy, W["ants"], W["iters"], 5, 2, stream, flush, barrier, dev)
    ms = statistics.mean(r["step_ms"])
    out = {"workload": "uniform1k", "n": W["n"], "ants": W["ants"], "iterations": W["iters"], "metric": METRIC,
           "unit": UNIT, "value": W["ants"] * W["iters"] / (ms / 1e3), "ms_per_step": ms, "steps": 5,
           "best_length": r["best_length"]}
    if not args.no_cpu:
        import oracle

        res = {}
        for th in (1, host_cores()):
            t0 = time.perf_counter()
            col = oracle.Colony(xy, 16, threads=th)
            col.iterate(W["ants"], W["iters"])
            L = col.best()[1]
            col.close()
            res[th] = (time.perf_counter() - t0, L)
        t1, tn = res[1][0], res[host_cores()][0]
        out["cpu_baseline"] = {
            "value": W["ants"] * W["iters"] / tn, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
            "extrapolated": False, "sample": "the whole workload (set-up + 32 ants x 200 iterations), measured",
            "single_thread": {"ant_solutions_per_s": W["ants"] * W["iters"] / t1, "cores": 1, "seconds": t1},
            "all_cores": {"ant_solutions_per_s": W["ants"] * W["iters"] / tn, "cores": host_cores(), "seconds": tn},
            "same_best_length_as_gpu": bool(res[1][1] == r["best_length"] == res[host_cores()][1])}
    return out


def bench_stippled200k(args, stream, flush, barrier, dev, peak, peak_src, l2_peak):
    """The n = 200,000 workload (2,048 ants, 50 iterations): full solves on
    the GPU with the per-ant kernel's roofline, and an oracle sample."""
    from paper_2203_02228_gb300 import inputs

    W = inputs.WORKLOADS["stippled200k"]
    xy = inputs.workload_points("stippled200k")
    n, ants, iters = xy.shape[0], W["ants"], W["iters"]
    r = bench_colony(xy, ants, iters, args.c3_steps, 1, stream, flush, barrier, dev)
    ms = statistics.mean(r["step_ms"])
    out = {"workload": "stippled200k", "n": n, "ants": ants, "iterations": iters, "metric":
           "ant-solutions/sec at 200k nodes", "unit": UNIT, "value": ants * iters / (ms / 1e3), "ms_per_step": ms,
           "steps": args.c3_steps, "gpu_launches": r["launches"], "best_length": r["best_length"],
           "roofline": roofline_line("k_ants_blk<16> (construction + local search)", n, ants, iters, r["ants_ms"],
                                     r["ants_launches"], r["algo_bytes"], peak, peak_src, l2_peak)}
    if not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline_line(xy, ants, iters, 16, host_cores())
    return out


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
    from paper_2203_02228_gb300 import tuner_report

    tuned = [r for r in tuner_report() if r["goal"] == "batch" and r["ants"] == ants]

    # the same batch with every colony on segment tables (no tuner), timed
    # the same way, to show what the tuner's choice is worth
    def run_fixed(mode):
        b = Batch(xs, k, seeds=seeds, stream=stream)
        b.set_plan(mode)
        b.iterate(ants, iters)
        tours, lens = b.tours()
        b.close()
        return lens

    run_fixed(0)
    flush.zero_()
    barrier()
    t0 = time.perf_counter()
    lens_tab = run_fixed(0)
    t_tab = time.perf_counter() - t0

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
        "tuner_ms_per_class": tuned,
        "all_segment_tables": {"value": len(xs) / t_tab, "unit": "instances/s", "seconds": t_tab,
                               "equal_lengths": bool(np.array_equal(lens_tab, lens))},
        "gpu_launches_per_batch": int(launches), "graph_launches_per_batch": 1, "cpu_baseline": cpu,
        "h2d_bytes_per_batch": int(8 * ns.sum()), "d2h_bytes_per_batch": int(4 * ns.sum() + 8 * len(xs)),
    }


def serve_plan(rates, requests):
    """Requests per rate: `requests` where the stream saturates the GPU,
    fewer at the lowest rates so that each trace arrives within ~30 s."""
    return [(r, int(min(requests, max(30, round(30 * r))))) for r in rates]


def plain_loop_times(arrivals, service):
    """First-come-first-served completion times of one instance at a time:
    C_i = max(A_i, C_{i-1}) + S_i."""
    done, t = [], 0.0
    for a_i, s_i in zip(arrivals, service):
        t = max(t, a_i) + s_i
        done.append(t)
    return np.array(done)


def bench_served(args, stream, barrier):
    """Poisson streams of requests (n log-uniform in [1e3, 1e5], 256 ants,
    50 iterations) through the server -- admission by device memory,
    continuous batching -- at each rate, and the plain loop (one Colony at
    a time, first come first served) on the same traces.  Time-to-budget =
    completion - arrival, host clock.  The plain loop's service time of
    each request is measured once (each instance solved alone, one after
    another on the idle GPU, through the public API); its completions on a
    trace follow from the arrivals by the FCFS recursion."""
    import threading as th

    from paper_2203_02228_gb300 import Colony, Server, inputs

    w = inputs.SERVE_WORKLOADS["serve100k"]
    plan = serve_plan(args.serve_rates, args.serve_requests)
    nmax = max(c for _, c in plan)
    xs, seeds, _ = inputs.serve_trace("serve100k", nmax, 1.0)
    out = {"workload": "serve100k", "ants": w["ants"], "iterations": w["iters"], "k": w["k"],
           "n_range": [w["lo"], w["hi"]], "metric": "time-to-budget p50/p99 (s), instances/sec",
           "pool_bytes": args.serve_pool_gb << 30, "rates": []}
    # warm: kernel tuner and module load, outside the timed streams
    with Server(1 << 30) as s:
        for j, n in enumerate((1500, 6000, 30000)):
            s.wait(s.submit(inputs.uniform(n, seed=j), w["k"], w["ants"], 2, 1))
    # plain loop: each request alone, once
    barrier()
    service, plens = [], []
    for i, x in enumerate(xs):
        t0 = time.perf_counter()
        c = Colony(x, w["k"], seed=int(seeds[i]), stream=stream)
        c.iterate(w["ants"], w["iters"])
        _, L = c.best()
        c.close()
        service.append(time.perf_counter() - t0)
        plens.append(L)
    out["plain_service_s"] = {"mean": float(np.mean(service)), "p50": float(np.median(service)),
                              "max": float(np.max(service)), "requests": len(service)}
    for rate, count in plan:
        _, _, arr = inputs.serve_trace("serve100k", count, rate)
        barrier()
        with Server(args.serve_pool_gb << 30) as s:
            t0 = time.perf_counter()
            tickets = [None] * count

            def feed():
                for i in range(count):
                    d = t0 + arr[i] - time.perf_counter()
                    if d > 0:
                        time.sleep(d)
                    tickets[i] = s.submit(xs[i], w["k"], w["ants"], w["iters"], int(seeds[i]))

            f = th.Thread(target=feed)
            f.start()
            f.join()
            res = [s.wait(t) for t in tickets]
            st = s.stats()
        lat = np.array([(r[3] - r[2]) / 1e9 for r in res])
        span = (max(r[3] for r in res) - min(r[2] for r in res)) / 1e9
        served = {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                  "mean_s": float(lat.mean()), "instances_per_s": count / span,
                  "ant_solutions_per_s": count * w["ants"] * w["iters"] / span,
                  "peak_active": st["peak_active"], "rounds": st["rounds"],
                  "gpu_launches": st["kernel_launches"], "mean_best_length": float(np.mean([r[1] for r in res]))}
        done = plain_loop_times(arr, service[:count])
        plat = done - arr
        plain = {"p50_s": float(np.percentile(plat, 50)), "p99_s": float(np.percentile(plat, 99)),
                 "mean_s": float(plat.mean()), "instances_per_s": count / (done[-1] - arr[0])}
        out["rates"].append({"rate_per_s": rate, "requests": count, "served": served, "plain_loop": plain,
                             "equal_lengths": bool(np.array_equal([r[1] for r in res], plens[:count]))})
    if not args.no_cpu:
        # the oracle on three requests of the trace (10th, 50th, 90th size
        # percentile): set-up + 1 iteration of 32 ants, scaled to 256 ants x 50
        import oracle

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
                               "kind": "oracle", "extrapolated": True,
                               "sample": "3 requests (10th/50th/90th size percentile, n = %s): oracle set-up + 1 "
                               "iteration of 32 ants measured, scaled to %d ants x %d iterations; one request "
                               "at a time" % ([int(ns[i]) for i in pick], w["ants"], w["iters"])}
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
    ap.add_argument("--ref-ants", type=int, default=128, help="ants per step of the reference arm")
    ap.add_argument("--ref-warm-iters", type=int, default=8)
    ap.add_argument("--iters", type=int, default=0, help="override the iteration budget (testing only)")
    ap.add_argument("--sections", default="main,uniform1k,stippled200k,batch,serve",
                    help="comma list of: main, uniform1k, stippled200k, batch, serve")
    ap.add_argument("--c3-steps", type=int, default=2)
    ap.add_argument("--batch-steps", type=int, default=3)
    ap.add_argument("--serve-rates", type=float, nargs="+", default=[1, 2, 5, 10, 20, 50, 100, 200])
    ap.add_argument("--serve-requests", type=int, default=100)
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

    from paper_2203_02228_gb300 import build, l2_probe

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    peak, peak_src = load_peaks()
    l2_peak = max(l2_probe(48 << 20, 200) for _ in range(3))
    extra = {}

    if "main" not in sections:
        if "uniform1k" in sections:
            extra["uniform1k"] = bench_uniform1k(args, stream, flush, barrier, dev)
        if "stippled200k" in sections:
            extra["stippled200k"] = bench_stippled200k(args, stream, flush, barrier, dev, peak, peak_src, l2_peak)
        if "batch" in sections:
            extra["batched"] = bench_batched(args, stream, flush, barrier)
        if "serve" in sections:
            extra["served"] = bench_served(args, stream, barrier)
        if rank == 0:
            print(json.dumps(extra), flush=True)
        return

    xy = inputs.workload_points(args.workload)
    n, ants, iters = xy.shape[0], W["ants"], W["iters"]

    clocks = ClockSampler(local)
    clocks.start()
    r = bench_colony(xy, ants, iters, args.steps, args.warmup, stream, flush, barrier, dev)
    barrier()
    clk = clocks.stop()

    ms = max_over_ranks(statistics.mean(r["step_ms"]), world, dev)
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
        for _ in range(max(1, min(args.steps, 5))):
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

    roofline = roofline_line("k_ants_blk<16> (construction + local search)", n, ants, iters, r["ants_ms"],
                             r["ants_launches"], r["algo_bytes"], peak, peak_src, l2_peak,
                             recorded_traffic() if args.workload == "stippled100k" else None)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline_line(xy, ants, iters, 16, host_cores())

    if world == 1:
        if "uniform1k" in sections:
            extra["uniform1k"] = bench_uniform1k(args, stream, flush, barrier, dev)
        if "stippled200k" in sections:
            extra["stippled200k"] = bench_stippled200k(args, stream, flush, barrier, dev, peak, peak_src, l2_peak)
        if "batch" in sections:
            extra["batched"] = bench_batched(args, stream, flush, barrier)
        if "serve" in sections:
            extra["served"] = bench_served(args, stream, barrier)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+int64", "data": "synthetic",
            "config": {"workload": args.workload, "n": n, "ants": ants, "iterations": iters, "k": 16,
                       "seed": 1, "l2": "flushed before every step (512 MB write)",
                       "parallelism": "independent colonies per rank" if world > 1 else "single colony"},
            "e2e": e2e, "gpu_launches": r["launches"], "roofline": roofline, "cpu_baseline": cpu,
            "clocks": clk,
        }
        line.update(extra)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
