"""Batched colonies (include/faco_batch.h) vs. the one-colony path and the
CPU oracle (needs a GB300).

Colony i of a batch must equal, bit for bit, the colony that faco_create_ex
builds for the same instance and seed, driven by the same iterate calls:
global-best tour and length, pheromone, counters.  Every kernel plan gives
the same results.  Sampled colonies of the full 512-instance workload are
checked against the oracle directly.
"""
import numpy as np
import pytest

import oracle
from paper_2203_02228_gb300 import Batch, Colony, inputs

pytestmark = pytest.mark.gpu


def mixed_instances():
    """Uneven sizes, two point distributions, and the degenerate n = 3, 4, 9."""
    sizes = [200, 3, 1300, 4, 9, 517, 2600, 257, 4100]
    xs = []
    for j, n in enumerate(sizes):
        if n <= 16:
            xs.append(inputs.uniform(n, seed=500 + j, side=1000))
        elif j % 2:
            xs.append(inputs.stippled(n, seed=600 + j, blobs=6, ridges=1, side=50_000))
        else:
            xs.append(inputs.uniform(n, seed=500 + j))
    return xs


def same_bits(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


ALGO_COUNTERS = ("iteration", "best_length", "initial_length", "source_length", "aco_steps", "new_edges",
                 "backup_picks", "global_picks", "ls_pops", "moves_2opt", "moves_or")


@pytest.mark.parametrize("plan", [None, 0, 1, 2, 3], ids=["tuned", "tables", "arrays2", "arrays4", "arrays8"])
def test_batch_equals_single_colonies(plan):
    xs = mixed_instances()
    seeds = (np.arange(len(xs), dtype=np.uint64) * 7919 + 3)
    b = Batch(xs, 16, seeds=seeds, plan=plan)
    b.iterate(12, 4)
    b.iterate(12, 3)  # a second budget: a second graph
    tours, lens = b.tours()
    assert np.all(b.plan() >= 0)
    for i, xy in enumerate(xs):
        c = Colony(xy, 16, seed=int(seeds[i]))
        c.iterate(12, 4)
        c.iterate(12, 3)
        t, L = c.best()
        assert lens[i] == L, i
        np.testing.assert_array_equal(tours[i], t, err_msg="colony %d" % i)
        bt, bL = b.best(i)
        assert bL == L
        np.testing.assert_array_equal(bt, t)
        assert same_bits(b.tau(i), c.tau()), i
        bs, cs = b.stats(i), c.stats()
        for f in ALGO_COUNTERS:
            assert getattr(bs, f) == getattr(cs, f), (i, f)
        c.close()


def test_batch_plans_agree_and_match_oracle():
    xs = mixed_instances()[:6]
    seeds = np.arange(11, 17, dtype=np.uint64)
    res = []
    for plan in (0, 1, 3, -1):
        b = Batch(xs, 16, seeds=seeds, plan=plan)
        b.iterate(10, 6)
        res.append((b.tours(), [b.tau(i) for i in range(len(xs))]))
        b.close()
    for (tours, lens), taus in res[1:]:
        np.testing.assert_array_equal(lens, res[0][0][1])
        for i in range(len(xs)):
            np.testing.assert_array_equal(tours[i], res[0][0][0][i])
            assert same_bits(taus[i], res[0][1][i])
    # the oracle, directly, for every colony
    (tours, lens), taus = res[0]
    for i, xy in enumerate(xs):
        o = oracle.Colony(xy, 16, seed=int(seeds[i]), threads=8)
        o.iterate(10, 6)
        ot, oL = o.best()
        assert lens[i] == oL
        np.testing.assert_array_equal(tours[i], ot)
        assert same_bits(taus[i], o.tau())


def test_batch_k32_and_no_backup():
    xs = [inputs.uniform(n, seed=70 + n) for n in (40, 333, 900)]
    b = Batch(xs, 32, bl_size=0, seeds=[5, 6, 7])
    b.iterate(8, 5)
    tours, lens = b.tours()
    for i, xy in enumerate(xs):
        c = Colony(xy, 32, bl_size=0, seed=5 + i)
        c.iterate(8, 5)
        t, L = c.best()
        assert lens[i] == L
        np.testing.assert_array_equal(tours[i], t)
        assert same_bits(b.tau(i), c.tau())


def test_batch_without_seeds_uses_params_seed():
    xs = [inputs.uniform(300, seed=1), inputs.uniform(450, seed=2)]
    b = Batch(xs, 16, seed=99)
    b.iterate(6, 4)
    for i, xy in enumerate(xs):
        c = Colony(xy, 16, seed=99)
        c.iterate(6, 4)
        assert b.best(i)[1] == c.best()[1]
        np.testing.assert_array_equal(b.best(i)[0], c.best()[0])


def test_batch512_full_workload_sampled_against_oracle():
    """The 512-instance workload in the benchmark's launch configuration (64
    ants, 100 iterations, one graph): tours are permutations with their
    stated lengths; sampled colonies (smallest, largest, three others) equal
    the oracle bit for bit."""
    w = inputs.BATCH_WORKLOADS["batch512"]
    xs, seeds = inputs.batch_workload("batch512")
    b = Batch(xs, w["k"], seeds=seeds)
    b.iterate(w["ants"], w["iters"])
    tours, lens = b.tours()
    for i, xy in enumerate(xs):
        t = tours[i]
        assert np.array_equal(np.sort(t), np.arange(xy.shape[0]))
        assert lens[i] == oracle.tour_length(xy, t)
    ns = np.array([x.shape[0] for x in xs])
    sample = sorted({int(np.argmin(ns)), int(np.argmax(ns)), 7, 200, 401})
    for i in sample:
        o = oracle.Colony(xs[i], w["k"], seed=int(seeds[i]), threads=16)
        o.iterate(w["ants"], w["iters"])
        ot, oL = o.best()
        assert lens[i] == oL, i
        np.testing.assert_array_equal(tours[i], ot)
        assert same_bits(b.tau(i), o.tau()), i


def test_batch_base_faco():
    """Base FACO (no local search on new tours) in a batch equals the
    one-colony path, for both kernel families."""
    xs = mixed_instances()[:5]
    for plan in (0, 3):
        b = Batch(xs, 16, seeds=[21, 22, 23, 24, 25], plan=plan, local_search=0, rho=0.9, min_new_edges=40)
        b.iterate(10, 5)
        tours, lens = b.tours()
        for i, xy in enumerate(xs):
            c = Colony(xy, 16, seed=21 + i, local_search=0, rho=0.9, min_new_edges=40)
            c.iterate(10, 5)
            t, L = c.best()
            assert lens[i] == L, (plan, i)
            np.testing.assert_array_equal(tours[i], t)
            assert same_bits(b.tau(i), c.tau())


def test_initial_search_with_positions_in_global_memory():
    """A batch whose largest colony is too large for the initial search's
    shared-memory positions runs every colony's initial search on positions
    in global memory; the small colonies must still equal their one-colony
    runs, which keep the positions in shared memory."""
    xs = [inputs.uniform(120_000, seed=71), inputs.uniform(900, seed=72), inputs.stippled(2000, seed=73, blobs=4,
                                                                                           ridges=1, side=60_000)]
    seeds = np.array([5, 6, 7], dtype=np.uint64)
    b = Batch(xs, 16, seeds=seeds)
    b.iterate(8, 1)
    tours, lens = b.tours()
    for i in (1, 2):
        c = Colony(xs[i], 16, seed=int(seeds[i]))
        c.iterate(8, 1)
        t, L = c.best()
        assert lens[i] == L, i
        np.testing.assert_array_equal(tours[i], t)
        assert b.stats(i).initial_length == c.stats().initial_length


def test_batch_initial_tours_with_three_opt():
    """Batched set-up with init_3opt: every colony's initial tour equals the
    oracle's (one block per colony, the same search)."""
    xs = mixed_instances()
    seeds = np.arange(11, 11 + len(xs), dtype=np.uint64)
    b = Batch(xs, 16, seeds=seeds, init_3opt=1)
    b.iterate(8, 2)
    for i, xy in enumerate(xs):
        o = oracle.Colony(xy, 16, seed=int(seeds[i]), init_3opt=1, threads=4)
        o.iterate(8, 2)
        t, L = b.best(i)
        assert L == o.best()[1]
        np.testing.assert_array_equal(t, o.best()[0])
        assert b.stats(i).initial_length == o.initial()[1]
