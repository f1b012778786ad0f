"""The seeded input recipes (paper_2203_02228_gb300/inputs.py) have the
properties the parity tests and the benchmark rely on: integer points in
range, all distinct (so every distance between distinct nodes is positive),
the same points for the same seed, the stated sizes, and for the stippled
stand-in a clustered density rather than a uniform one."""
import numpy as np
import pytest

from paper_2203_02228_gb300 import inputs


def distinct(xy):
    return len(np.unique(xy[:, 0].astype(np.int64) * (1 << 32) + xy[:, 1])) == len(xy)


@pytest.mark.parametrize("gen", [lambda s: inputs.uniform(5000, seed=s, side=20_000),
                                 lambda s: inputs.stippled(5000, seed=s, blobs=8, ridges=2, side=20_000)],
                         ids=["uniform", "stippled"])
def test_points_in_range_distinct_and_reproducible(gen):
    a, b, c = gen(11), gen(11), gen(12)
    assert a.dtype == np.int32 and a.shape == (5000, 2)
    assert a.min() >= 0 and a.max() < 20_000
    assert distinct(a)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, c)


def test_dense_draws_still_distinct():
    # 600 points on a 30 x 30 lattice: two thirds of the sites, duplicates
    # redrawn until none is left
    xy = inputs.uniform(600, seed=3, side=30)
    assert distinct(xy) and len(xy) == 600
    with pytest.raises(ValueError):
        inputs.uniform(901, seed=3, side=30)


def test_stippled_is_clustered():
    # occupancy of a coarse grid: the stippled points crowd into fewer cells
    # than uniform points do
    side, n, cells = 100_000, 20_000, 32
    occ = []
    for xy in (inputs.uniform(n, seed=5, side=side), inputs.stippled(n, seed=5, blobs=16, ridges=2, side=side)):
        h, _, _ = np.histogram2d(xy[:, 0], xy[:, 1], bins=cells, range=[[0, side], [0, side]])
        occ.append(h.ravel())
    # uniform: Poisson counts, coefficient of variation about 1/sqrt(mean)
    cv_uniform, cv_stippled = (o.std() / o.mean() for o in occ)
    assert cv_uniform < 2 / np.sqrt(n / cells ** 2)
    assert cv_stippled > 3 * cv_uniform
    assert (occ[1] == 0).sum() > (occ[0] == 0).sum()


def test_benchmark_workload_shape():
    w = inputs.WORKLOADS["stippled100k"]
    assert (w["n"], w["ants"], w["iters"]) == (100_000, 1024, 100)
    xy = inputs.workload_points("stippled100k")
    assert xy.shape == (100_000, 2) and xy.max() < w["side"] and distinct(xy)


def test_batch_sizes_are_log_uniform():
    n = inputs.batch_sizes(4096, seed=4000, lo=200, hi=20_000)
    assert n.min() >= 200 and n.max() <= 20_000
    # log-uniform: the median sits near the geometric mean, quartiles near
    # the quarter points in log space
    lq = np.log(n)
    lo, hi = np.log(200), np.log(20_000)
    for q, f in ((25, 0.25), (50, 0.5), (75, 0.75)):
        assert abs(np.percentile(lq, q) - (lo + f * (hi - lo))) < 0.1
    xs, seeds = inputs.batch_workload("batch512")
    assert len(xs) == 512 and list(seeds[:3]) == [1, 2, 3]
    assert [x.shape[0] for x in xs[:8]] == list(inputs.batch_sizes(512, seed=4000)[:8])


def test_serve_trace_is_a_poisson_stream():
    xs, seeds, arr = inputs.serve_trace("serve100k", 400, rate=8.0)
    assert len(xs) == len(seeds) == len(arr) == 400
    assert arr[0] == 0.0 and np.all(np.diff(arr) >= 0)
    gaps = np.diff(arr)
    assert abs(gaps.mean() - 1 / 8.0) < 0.02
    # exponential gaps: the coefficient of variation is near 1
    assert 0.8 < gaps.std() / gaps.mean() < 1.2
    ns = np.array([x.shape[0] for x in xs])
    assert ns.min() >= 1000 and ns.max() <= 100_000
