"""Pins for the oracle's primitives, each against something other than itself.

* EUC_2D (Sec. 2.1 cost d_ij, TSPLIB rounding): Python's exact ``math.isqrt``.
* Philox4x32-10: the published known-answer vectors (tests/golden).
* Roulette of Eq. 1: frequencies over a dense grid of uniforms against the
  proportions tau*eta / sum; zero weights are never picked.
* Candidate/backup lists (Sec. 4.1): numpy lexsort over the full distance row.
* Nearest-neighbour initial tour (Sec. 4.3): the textbook heuristic by brute
  force -- with sorted candidate/backup lists the first unvisited list entry is
  always the globally nearest unvisited node, for any list lengths.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2203_02228_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def exact_round_sqrt(m: int) -> int:
    # floor(sqrt(m) + 1/2) = floor((floor(2 sqrt(m)) + 1) / 2), exact in integers
    return (math.isqrt(4 * m) + 1) // 2


def test_isqrt_exhaustive_small():
    for m in range(0, 1 << 16):
        assert oracle.isqrt(m) == math.isqrt(m)


def test_isqrt_random_large():
    rng = np.random.default_rng(7)
    vals = list(rng.integers(0, 1 << 62, size=4000, dtype=np.int64)) + \
        [r * r + d for r in (1 << 20, (1 << 24) + 3, 3037000499) for d in (-1, 0, 1)]
    for m in vals:
        m = int(m)
        if m < 0:
            continue
        assert oracle.isqrt(m) == math.isqrt(m)


def test_euc2d_matches_exact_rounding():
    rng = np.random.default_rng(11)
    xy = rng.integers(0, 1 << 24, size=(2000, 2)).astype(np.int32)
    for i in range(0, 2000, 2):
        dx = int(xy[i, 0]) - int(xy[i + 1, 0])
        dy = int(xy[i, 1]) - int(xy[i + 1, 1])
        assert oracle.euc2d(xy, i, i + 1) == exact_round_sqrt(dx * dx + dy * dy)
    # near-half cases: m = r^2 + r (just below r + 1/2) and r^2 + r + 1 (above)
    for r in (1, 2, 3, 1000, 99999, 1 << 20):
        for m, want in ((r * r + r, r), (r * r + r + 1, r + 1)):
            assert exact_round_sqrt(m) == want
    # the TSPLIB nint(sqrt()) form agrees where double sqrt is exact enough
    pts = np.array([[0, 0], [3, 4], [1, 1], [10, 0], [7, 7]], np.int32)
    for a in range(5):
        for b in range(5):
            dx, dy = pts[a] - pts[b]
            assert oracle.euc2d(pts, a, b) == int(math.sqrt(float(dx * dx + dy * dy)) + 0.5)


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(t, 16) for t in line.split()])
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox(r[0:4], r[4:6])
        assert [int(x) for x in out] == r[6:10]


def test_draw_layout_and_u01():
    # draw idx uses counter word idx % 4 of block idx // 4
    seed = 0x123456789ABCDEF
    for idx in range(12):
        block = oracle.philox([idx >> 2, 5, 9, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert oracle.draw(seed, idx, 5, 9, 0) == int(block[idx & 3])
    for x in (0, 1, 255, 256, 0xFFFFFFFF, 0x80000000):
        assert oracle.u01(x) == (x >> 8) / float(1 << 24)
    assert oracle.u01(0xFFFFFFFF) < 1.0


def test_start_node_is_uniform():
    n, cnt = 37, 37000
    hits = np.zeros(n)
    for a in range(cnt):
        x = oracle.draw(1, 0, a, 1, 0)
        hits[(x * n) >> 32] += 1
    chi2 = ((hits - cnt / n) ** 2 / (cnt / n)).sum()
    assert chi2 < 80  # 36 dof; p ~ 1e-4 threshold


def test_roulette_proportions():
    rng = np.random.default_rng(3)
    for trial in range(6):
        w = rng.random(16).astype(np.float32)
        w[rng.random(16) < 0.3] = 0.0
        if not (w > 0).any():
            w[5] = 1.0
        grid = 1 << 14
        hits = np.zeros(16)
        for i in range(grid):
            s = oracle.roulette(w, (i + 0.5) / grid)
            assert w[s] > 0
            hits[s] += 1
        np.testing.assert_allclose(hits / grid, w / w.sum(), atol=2.0 / grid + 1e-6)


def test_roulette_edge_cases():
    one = np.zeros(16, np.float32)
    one[7] = 0.25
    for u in (0.0, 0.5, 0.999999940):
        assert oracle.roulette(one, u) == 7
    # u -> 1 must still pick a positive weight (rounding of r = u * total)
    rng = np.random.default_rng(5)
    for _ in range(2000):
        w = (rng.random(16) * 10.0 ** rng.uniform(-30, 10)).astype(np.float32)
        w[rng.random(16) < 0.5] = 0
        if not (w > 0).any():
            continue
        s = oracle.roulette(w, float(np.nextafter(np.float32(1), np.float32(0))))
        assert w[s] > 0


def test_roulette_zero_padding_to_32_is_equivalent():
    # width 32 with zeros in slots 16..31 gives the same pick as width 16
    rng = np.random.default_rng(9)
    L = oracle.lib()
    for _ in range(3000):
        w = rng.random(16).astype(np.float32)
        w[rng.random(16) < 0.4] = 0
        if not (w > 0).any():
            continue
        u = np.float32(rng.random())
        w32 = np.zeros(32, np.float32)
        w32[:16] = w
        a = L.orc_roulette(np.ascontiguousarray(w), 16, float(u))
        b = L.orc_roulette(w32, 32, float(u))
        assert a == b


def _brute_knn(xy, K):
    xy = xy.astype(np.int64)
    n = len(xy)
    out = np.zeros((n, K), np.int32)
    idx = np.arange(n)
    for u in range(n):
        m = ((xy - xy[u]) ** 2).sum(1)
        order = np.lexsort((idx, m))
        order = order[order != u]
        out[u] = order[:K]
    return out


@pytest.mark.parametrize("kind", ["uniform", "lattice", "stippled"])
def test_knn_matches_lexsort(kind):
    if kind == "uniform":
        xy = inputs.uniform(700, seed=21, side=5000)
    elif kind == "lattice":
        xy = inputs.lattice(20, 25, step=3)
    else:
        xy = inputs.stippled(900, seed=22, blobs=8, ridges=2, side=20000)
    K = 80
    np.testing.assert_array_equal(oracle.knn_rows(xy, K), _brute_knn(xy, K))


def _nn_textbook(xy):
    xy = xy.astype(np.int64)
    n = len(xy)
    vis = np.zeros(n, bool)
    route = [0]
    vis[0] = True
    idx = np.arange(n)
    for _ in range(n - 1):
        u = route[-1]
        m = ((xy - xy[u]) ** 2).sum(1)
        m = np.where(vis, np.iinfo(np.int64).max, m)
        order = np.lexsort((idx, m))
        route.append(int(order[0]))
        vis[order[0]] = True
    return np.array(route, np.int32)


@pytest.mark.parametrize("k,bl", [(2, 0), (3, 2), (5, 10), (16, 64)])
def test_nn_tour_is_textbook_nearest_neighbour(k, bl):
    xy = inputs.uniform(400, seed=31 + k, side=100000)
    nn = oracle.knn_rows(xy, k + bl)
    got = oracle.nn_tour(xy, nn[:, :k], nn[:, k:k + bl])
    np.testing.assert_array_equal(got, _nn_textbook(xy))
