"""GPU path vs. the CPU oracle, element by element (needs a GB300).

Integer results (lists, tours, lengths, history) must be bit-exact; the FP32
pheromone too (the library and the oracle take the same IEEE operations in the
same order: products tau*eta, the Kogge-Stone scan, fmaf in Eq. 2), so the
tolerance asked for (1e-6 relative) is checked and bit equality asserted.
Inputs are seeded and synthetic (paper_2203_02228_gb300.inputs).
"""
import numpy as np
import pytest

import oracle
from paper_2203_02228_gb300 import Colony, device_selftest, inputs

pytestmark = pytest.mark.gpu

TAU_RTOL = 1e-6


def make_pair(xy, k=16, **kw):
    g = Colony(xy, k, keep_ant_tours=1, keep_pre_ls=1, **kw)
    o = oracle.Colony(xy, k, keep_pre_ls=1, threads=8, **kw)
    return g, o


def assert_tau(g, o):
    tg, to = g.tau(), o.tau()
    np.testing.assert_allclose(tg, to, rtol=TAU_RTOL, atol=0)
    assert np.array_equal(tg.view(np.uint32), to.view(np.uint32))


def assert_same_state(g, o, ants):
    np.testing.assert_array_equal(g.lists()[0], o.lists()[0])
    assert g.best()[1] == o.best()[1]
    np.testing.assert_array_equal(g.best()[0], o.best()[0])
    np.testing.assert_array_equal(g.source()[0], o.source()[0])
    assert g.source()[1] == o.source()[1]
    assert_tau(g, o)
    np.testing.assert_array_equal(g.limits(), o.limits())


# ---- primitives ------------------------------------------------------------

def test_device_philox_matches_oracle():
    rng = np.random.default_rng(1)
    cnt = 4096
    inp = rng.integers(0, 1 << 32, size=(cnt, 4), dtype=np.uint64).astype(np.uint32)
    inp[:64, 0] = np.arange(64)
    out = np.zeros(cnt, np.uint32)
    seed = 0x0123456789ABCDEF
    device_selftest(0, inp, out, cnt, seed=seed)
    want = [oracle.draw(seed, *map(int, r)) for r in inp]
    np.testing.assert_array_equal(out, np.array(want, np.uint32))


def test_device_euc2d_matches_oracle():
    rng = np.random.default_rng(2)
    cnt = 60000
    inp = rng.integers(0, 1 << 24, size=(cnt, 4)).astype(np.int32)
    inp[:100] = rng.integers(0, 50, size=(100, 4))  # small distances and zeros
    inp[100:110] = [[0, 0, (1 << 24) - 1, (1 << 24) - 1]] * 10  # the largest distance
    # next to a half-integer: (dx, dy) = (k, isqrt(k) + t) puts dx^2 + dy^2
    # around k^2 + k, the boundary between rounding to k and to k + 1, for
    # costs from 1 to 2^24 (the library's fast path covers costs below ~10^6
    # and |dx|, |dy| < 2^22; the rest take the exact integer steps)
    k = np.unique(np.exp(rng.uniform(0, np.log((1 << 24) - 1), 8000)).astype(np.int64))
    near = []
    for t in (-1, 0, 1):
        dy = np.floor(np.sqrt(k.astype(np.float64))).astype(np.int64) + t
        ok = (dy >= 0) & (dy < (1 << 24))
        near.append(np.stack([np.zeros(ok.sum()), np.zeros(ok.sum()), k[ok], dy[ok]], 1))
    near = np.concatenate(near).astype(np.int32)
    near[1::2] = near[1::2][:, [2, 3, 0, 1]]  # both signs of dx, dy
    inp[200:200 + len(near)] = near
    # short edges in every direction around a point (the common case)
    inp[20000:30000, :2] = 5_000_000
    inp[20000:30000, 2:] = 5_000_000 + rng.integers(-3000, 3000, size=(10000, 2))
    out = np.zeros(cnt, np.int32)
    device_selftest(1, inp, out, cnt)
    want = [oracle.euc2d(np.array([[a, b], [c, d]], np.int32), 0, 1) for a, b, c, d in inp]
    np.testing.assert_array_equal(out, np.array(want, np.int32))


@pytest.mark.parametrize("width", [16, 32])
def test_device_roulette_matches_oracle(width):
    rng = np.random.default_rng(3 + width)
    cnt = 20000
    inp = np.zeros((cnt, width + 1), np.float32)
    w = (rng.random((cnt, width)) * 10.0 ** rng.uniform(-20, 5, size=(cnt, 1))).astype(np.float32)
    w[rng.random((cnt, width)) < 0.4] = 0
    w[:, 0] = np.where((w > 0).any(1), w[:, 0], 1.0)
    inp[:, :width] = w
    inp[:, width] = rng.random(cnt).astype(np.float32)
    inp[:50, width] = np.float32(np.nextafter(np.float32(1), np.float32(0)))
    out = np.zeros(cnt, np.int32)
    device_selftest(2, inp, out, cnt, width=width)
    L = oracle.lib()
    want = [L.orc_roulette(np.ascontiguousarray(inp[i, :width]), width, float(inp[i, width])) for i in range(cnt)]
    np.testing.assert_array_equal(out, np.array(want, np.int32))


# ---- set-up: lists and initial tour -----------------------------------------

@pytest.mark.parametrize("kind", ["uniform", "lattice", "stippled", "dups"])
def test_lists_and_initial_tour(kind):
    if kind == "uniform":
        xy = inputs.uniform(3000, seed=5)
    elif kind == "lattice":
        xy = inputs.lattice(40, 50, step=7)
    elif kind == "stippled":
        xy = inputs.stippled(4000, seed=6, blobs=12, ridges=3, side=50000)
    else:  # duplicate points: d = 0, eta = 1
        base = inputs.uniform(600, seed=7, side=2000)
        xy = np.concatenate([base, base[:50]])
    g = Colony(xy, 16)
    o = oracle.Colony(xy, 16, threads=8)
    gc, gb, ge = g.lists()
    oc, ob, oe = o.lists()
    np.testing.assert_array_equal(gc, oc)
    np.testing.assert_array_equal(gb, ob)
    assert np.array_equal(ge.view(np.uint32), oe.view(np.uint32))
    gi, gL = g.initial()
    oi, oL = o.initial()
    assert gL == oL
    np.testing.assert_array_equal(gi, oi)
    assert_tau(g, o)
    np.testing.assert_array_equal(g.limits(), o.limits())


# ---- iterations ------------------------------------------------------------

CASES = [
    # (name, n, ants, iters, k, extra params)
    ("uniform200", 200, 8, 25, 16, {}),
    ("stippled3000", 3000, 16, 30, 16, {}),
    ("no_oropt", 500, 12, 20, 16, dict(oropt=0)),
    ("no_verify", 500, 12, 20, 16, dict(verify_pass=0)),
    ("k32", 700, 8, 15, 32, {}),
    ("k5_bl0", 400, 8, 15, 5, dict(bl_size=0)),
    ("mmas_walk", 300, 6, 6, 8, dict(min_new_edges=1000, bl_size=4)),
    ("rho09_seed7", 800, 10, 20, 16, dict(rho=0.9, seed=7)),
    ("tiny9", 9, 4, 30, 16, {}),
    ("tiny4", 4, 3, 10, 16, {}),
    ("tiny3", 3, 2, 5, 16, {}),
    ("base_faco", 600, 12, 15, 16, dict(local_search=0, rho=0.9, min_new_edges=40)),
]


# Tour representation of the ants: "auto" = segment tables sized from shared
# memory, "arrays" = explicit route/pos for every ant, "tiny" = 8-segment
# tables, so that most ants overflow and are redone on arrays.
MODES = {"auto": -1, "arrays": 0, "tiny": 8}


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("name,n,ants,iters,k,extra", CASES, ids=[c[0] for c in CASES])
def test_iterations_bit_exact(name, n, ants, iters, k, extra, mode):
    if name.startswith("stippled"):
        xy = inputs.stippled(n, seed=n, blobs=10, ridges=2, side=60000)
    else:
        xy = inputs.uniform(n, seed=1000 + n, side=1_000_000 if n > 16 else 1000)
    g = Colony(xy, k, keep_ant_tours=1, keep_pre_ls=1, seg_cap=MODES[mode], **extra)
    o = oracle.Colony(xy, k, keep_pre_ls=1, threads=8, **extra)
    o_hist = []
    for it in range(iters):
        g.iterate(ants, 1)
        oh, o_al = o.iterate(ants, 1)
        o_hist.append(oh[0])
        gt, gl = g.ant_tours()
        ot, ol = o.ant_tours()
        np.testing.assert_array_equal(gl, o_al[0], err_msg="ant lengths, iteration %d" % (it + 1))
        gp, gpl, gchk = g.ant_pre()
        op, opl, ochk = o.ant_pre()
        np.testing.assert_array_equal(gp, op, err_msg="tours before LS, iteration %d" % (it + 1))
        np.testing.assert_array_equal(gpl, opl)
        for a in range(ants):
            np.testing.assert_array_equal(gchk[a], ochk[a])
        np.testing.assert_array_equal(gt, ot, err_msg="tours after LS, iteration %d" % (it + 1))
        assert_same_state(g, o, ants)
    np.testing.assert_array_equal(g.history(), np.array(o_hist))


def test_budget_in_one_call_equals_single_steps():
    xy = inputs.uniform(1500, seed=42)
    a = Colony(xy, 16)
    b = Colony(xy, 16)
    a.iterate(24, 30)
    for _ in range(30):
        b.iterate(24, 1)
    np.testing.assert_array_equal(a.history(), b.history())
    assert np.array_equal(a.tau().view(np.uint32), b.tau().view(np.uint32))
    np.testing.assert_array_equal(a.best()[0], b.best()[0])


def test_stippled20k_segments_bit_exact():
    """A mid-size clustered instance where the per-ant segment tables see
    hundreds of reversals: every ant length, the history and the state."""
    xy = inputs.stippled(20000, seed=2020, blobs=24, ridges=4, side=100_000)
    g = Colony(xy, 16, keep_ant_tours=1)
    o = oracle.Colony(xy, 16, threads=16)
    o_hist = []
    for it in range(12):
        g.iterate(48, 1)
        oh, oal = o.iterate(48, 1)
        o_hist.append(oh[0])
        np.testing.assert_array_equal(g.ant_tours()[1], oal[0], err_msg="iteration %d" % (it + 1))
    np.testing.assert_array_equal(g.history(), np.array(o_hist))
    assert_same_state(g, o, 48)
    st = g.stats()
    assert st.moves_2opt > 0 and st.moves_or > 0


def test_stippled100k_setup_and_first_iterations():
    """The n = 100,000 stippled workload at full size in the benchmark's
    launch configuration (1,024 ants): lists, initial tour, limits and the
    first two iterations of every ant, bit for bit."""
    xy = inputs.workload_points("stippled100k")
    g = Colony(xy, 16, keep_ant_tours=1)
    o = oracle.Colony(xy, 16, threads=16)
    gc, gb, ge = g.lists()
    oc, ob, oe = o.lists()
    np.testing.assert_array_equal(gc, oc)
    np.testing.assert_array_equal(gb, ob)
    assert np.array_equal(ge.view(np.uint32), oe.view(np.uint32))
    assert g.initial()[1] == o.initial()[1]
    np.testing.assert_array_equal(g.initial()[0], o.initial()[0])
    for it in range(2):
        g.iterate(1024, 1)
        oh, oal = o.iterate(1024, 1)
        gt, gl = g.ant_tours()
        np.testing.assert_array_equal(gl, oal[0])
        ot, _ = o.ant_tours()
        sample = np.arange(0, 1024, 97)
        np.testing.assert_array_equal(gt[sample], ot[sample])
    np.testing.assert_array_equal(g.history()[-1], oh[0])
    assert_same_state(g, o, 1024)


def test_uniform1k_full_workload_bit_exact():
    """The n = 1,000 workload in full: 32 ants x 200 iterations, seed 1."""
    xy = inputs.workload_points("uniform1k")
    g = Colony(xy, 16)
    o = oracle.Colony(xy, 16, threads=8)
    g.iterate(32, 200)
    oh, oal = o.iterate(32, 200)
    np.testing.assert_array_equal(g.history(), oh)
    assert_same_state(g, o, 32)


def test_stippled200k_setup_and_first_iterations():
    """The n = 200,000 stippled workload (256 blobs) at full size in the
    benchmark's launch configuration (2,048 ants): lists, initial tour
    (its local search keeps positions in global memory at this size),
    limits, and the first two iterations -- every ant's length, a sample
    of tours, the history and tau bits."""
    xy = inputs.workload_points("stippled200k")
    g = Colony(xy, 16, keep_ant_tours=1)
    o = oracle.Colony(xy, 16, threads=16)
    gc, gb, ge = g.lists()
    oc, ob, oe = o.lists()
    np.testing.assert_array_equal(gc, oc)
    np.testing.assert_array_equal(gb, ob)
    assert np.array_equal(ge.view(np.uint32), oe.view(np.uint32))
    assert g.initial()[1] == o.initial()[1]
    np.testing.assert_array_equal(g.initial()[0], o.initial()[0])
    np.testing.assert_array_equal(g.limits(), o.limits())
    o_hist = []
    for it in range(2):
        g.iterate(2048, 1)
        oh, oal = o.iterate(2048, 1)
        o_hist.append(oh[0])
        gt, gl = g.ant_tours()
        np.testing.assert_array_equal(gl, oal[0], err_msg="iteration %d" % (it + 1))
        ot, _ = o.ant_tours()
        sample = np.arange(3, 2048, 131)
        np.testing.assert_array_equal(gt[sample], ot[sample])
        del gt, ot
    np.testing.assert_array_equal(g.history(), np.array(o_hist))
    assert_same_state(g, o, 2048)
    assert g.stats().redone_ants >= 0


def test_one_colony_above_shared_position_limit():
    """n = 120,000 (stippled): the initial local search of a single colony
    keeps tour positions in global memory above ~106k nodes; its lists,
    initial tour and one iteration of 256 ants against the oracle."""
    xy = inputs.stippled(120_000, seed=1212, blobs=48, ridges=6, side=100_000)
    g = Colony(xy, 16, keep_ant_tours=1)
    o = oracle.Colony(xy, 16, threads=16)
    np.testing.assert_array_equal(g.lists()[0], o.lists()[0])
    assert g.initial()[1] == o.initial()[1]
    np.testing.assert_array_equal(g.initial()[0], o.initial()[0])
    g.iterate(256, 1)
    oh, oal = o.iterate(256, 1)
    np.testing.assert_array_equal(g.ant_tours()[1], oal[0])
    np.testing.assert_array_equal(g.history()[-1], oh[0])
    assert_same_state(g, o, 256)


# ---- the initial tour with 3-opt segment exchanges (init_3opt) --------------

@pytest.mark.parametrize("kind", ["uniform", "stippled", "lattice", "tiny"])
def test_initial_tour_with_three_opt(kind):
    """init_3opt = 1: the initial tour's search also tries the 3-opt
    segment exchange (Sec. 4.3); the tour, its length and the first
    iterations equal the oracle's."""
    if kind == "uniform":
        xy = inputs.uniform(2500, seed=15)
    elif kind == "stippled":
        xy = inputs.stippled(3000, seed=16, blobs=10, ridges=2, side=60_000)
    elif kind == "lattice":
        xy = inputs.lattice(30, 40, step=5)
    else:
        xy = inputs.uniform(12, seed=17, side=1000)
    g = Colony(xy, 16, init_3opt=1, keep_ant_tours=1)
    o = oracle.Colony(xy, 16, init_3opt=1, threads=8)
    gi, gL = g.initial()
    oi, oL = o.initial()
    assert gL == oL
    np.testing.assert_array_equal(gi, oi)
    plain = oracle.Colony(xy, 16, threads=8)
    if kind in ("uniform", "stippled"):
        assert plain.initial()[1] != oL  # the exchange changed the search's path
    g.iterate(16, 3)
    oh, _ = o.iterate(16, 3)
    np.testing.assert_array_equal(g.history(), oh)
    assert_same_state(g, o, 16)


def test_initial_tour_with_three_opt_above_shared_position_limit():
    """The same with tour positions in global memory (n = 110,000)."""
    xy = inputs.stippled(110_000, seed=1313, blobs=40, ridges=5, side=100_000)
    g = Colony(xy, 16, init_3opt=1)
    o = oracle.Colony(xy, 16, init_3opt=1, threads=16)
    assert g.initial()[1] == o.initial()[1]
    np.testing.assert_array_equal(g.initial()[0], o.initial()[0])


def test_stippled100k_steady_state():
    """The n = 100,000 workload past its first iterations (24 iterations of
    1,024 ants): the source has moved off the initial tour, searches run
    thousands of pops and the construction's nearest-unvisited searches
    take the block-wide path -- the whole history, every ant's length in
    the last iteration, and the final state equal the oracle's."""
    xy = inputs.workload_points("stippled100k")
    g = Colony(xy, 16, keep_ant_tours=1)
    o = oracle.Colony(xy, 16, threads=16)
    g.iterate(1024, 24)
    oh, oal = o.iterate(1024, 24)
    np.testing.assert_array_equal(g.history(), oh)
    np.testing.assert_array_equal(g.ant_tours()[1], oal[-1])
    assert_same_state(g, o, 1024)
    st = g.stats()
    assert st.global_picks > 0 and st.moves_or > 0
