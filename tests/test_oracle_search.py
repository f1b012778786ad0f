"""Pins for the oracle's search steps (construction, local search, pheromone).

Every expected value is computed here from first principles (explicit tour
surgery and full length recomputation, brute force over small instances),
never by retyping the oracle's formulas:

* Alg 3 (2-opt) with full neighbour lists and the verify pass ends in a tour
  that no 2-opt move of all O(n^2) improves; with Or-opt enabled no segment
  insertion of length 1..3 improves either.
* Local search never lengthens a tour and the returned gain equals the
  recomputed length difference.
* Alg 2 (focused construction): tours are permutations, the new edges
  relative to the source equal the counted ones (+ the closing edge), the
  checklist is exactly the heads of the new edges, the start node follows
  the Philox stream, after the quota every non-source edge is forced (both
  source neighbours already visited); with min_new_edges > n the walk is
  plain MMAS construction whose list fallbacks pick the nearest unvisited
  node.
* Eq. 2 with rho = 1/2 on a convex polygon (where the optimum is the hull
  tour and every ant returns it): source edges stay exactly at tau_max and
  other entries halve exactly each iteration until they reach tau_min.
* End to end: for n <= 9 the colony's best equals the exhaustive optimum.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from paper_2203_02228_gb300 import inputs


def dmat(xy):
    xy = np.asarray(xy, np.int64)
    n = len(xy)
    D = np.zeros((n, n), np.int64)
    for i in range(n):
        m = ((xy - xy[i]) ** 2).sum(1)
        D[i] = [(math.isqrt(4 * int(v)) + 1) // 2 for v in m]
    return D


def length(D, route):
    r = np.asarray(route)
    return int(D[r, np.roll(r, -1)].sum())


def best_2opt_delta(D, route):
    """Smallest length change over every 2-opt move (explicit reversal)."""
    n = len(route)
    L0 = length(D, route)
    best = 0
    for i in range(n - 1):
        for j in range(i + 2, n if i > 0 else n - 1):
            r = list(route)
            r[i + 1:j + 1] = r[i + 1:j + 1][::-1]
            best = min(best, length(D, r) - L0)
    return best


def best_oropt_delta(D, route):
    """Smallest change over moving a segment of 1..3 nodes (either
    orientation) between the ends of a tour edge not adjacent to it."""
    n = len(route)
    L0 = length(D, route)
    best = 0
    for i in range(n):
        for ell in (1, 2, 3):
            seg = [route[(i + t) % n] for t in range(ell)]
            rest = [route[(i + ell + t) % n] for t in range(n - ell)]  # q ... p
            p, q = rest[-1], rest[0]
            for t in range(len(rest)):
                u, v = rest[t], rest[(t + 1) % len(rest)]
                if u in (p, q) or v in (p, q):
                    continue
                for s in (seg, seg[::-1]):
                    r = rest[:t + 1] + s + rest[t + 1:]
                    best = min(best, length(D, r) - L0)
    return best


def is_perm(route, n):
    return sorted(int(x) for x in route) == list(range(n))


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("oropt", [0, 1])
def test_full_queue_ls_reaches_local_optimum(seed, oropt):
    n = 24 + 3 * seed
    xy = inputs.uniform(n, seed=100 + seed, side=10000)
    D = dmat(xy)
    cand = oracle.knn_rows(xy, n - 1)
    # start from the nearest-neighbour tour so that Alg 3's limit of n
    # applied moves is not what stops the search
    route = oracle.nn_tour(xy, cand[:, :4], cand[:, 4:8])
    L0 = length(D, route)
    out, gain, st = oracle.local_search(xy, cand, route, route.copy(), oropt=oropt, verify=1)
    assert st[oracle.ST_MOVES_2OPT] + st[oracle.ST_MOVES_OR] < n
    assert is_perm(out, n)
    assert length(D, out) == L0 - gain
    assert gain > 0
    assert best_2opt_delta(D, list(out)) == 0
    if oropt:
        assert best_oropt_delta(D, list(out)) == 0


@pytest.mark.parametrize("seed", range(4))
def test_ls_with_short_lists_never_lengthens(seed):
    n = 300
    xy = inputs.stippled(n, seed=200 + seed, blobs=6, ridges=1, side=20000)
    D = dmat(xy)
    cand = oracle.knn_rows(xy, 5)
    rng = np.random.default_rng(seed)
    route = rng.permutation(n).astype(np.int32)
    for oropt in (0, 1):
        for verify in (0, 1):
            q = rng.choice(n, size=40, replace=False).astype(np.int32)
            out, gain, st = oracle.local_search(xy, cand, route, q, oropt=oropt, verify=verify)
            assert is_perm(out, n)
            assert gain >= 0
            assert length(D, out) == length(D, route) - gain
            assert st[oracle.ST_MOVES_2OPT] + st[oracle.ST_MOVES_OR] <= n


def edge_set(route):
    r = list(route)
    return {frozenset((r[i], r[(i + 1) % len(r)])) for i in range(len(r))}


def check_construction(xy, C, src, pre, checks, it, seed, min_new):
    n = len(xy)
    pos_src = np.empty(n, np.int64)
    pos_src[src] = np.arange(n)
    E_src = edge_set(src)
    for a in range(pre.shape[0]):
        r = [int(x) for x in pre[a]]
        assert is_perm(r, n)
        assert r[0] == (oracle.draw(seed, 0, a, it, 0) * n) >> 32
        heads, new_idx = [], []
        for i in range(n - 1):
            if frozenset((r[i], r[i + 1])) not in E_src:
                heads.append(r[i + 1])
                new_idx.append(i)
        closing_new = frozenset((r[-1], r[0])) not in E_src
        assert list(checks[a]) == heads
        assert len(edge_set(r) - E_src) == len(heads) + int(closing_new)
        if len(heads) < min_new:
            continue  # tour completed before the quota
        # after the quota, every non-source edge is forced
        seen = set(r[:new_idx[min_new - 1] + 2])
        for i in range(new_idx[min_new - 1] + 1, n - 1):
            if frozenset((r[i], r[i + 1])) not in E_src:
                x = r[i]
                assert src[(pos_src[x] + 1) % n] in seen and src[(pos_src[x] - 1) % n] in seen
            seen.add(r[i + 1])


@pytest.mark.parametrize("kind,n,seed", [("uniform", 200, 1), ("stippled", 400, 7), ("uniform", 57, 3)])
def test_focused_construction_invariants(kind, n, seed):
    xy = inputs.uniform(n, seed=300 + n) if kind == "uniform" else \
        inputs.stippled(n, seed=300 + n, blobs=5, ridges=1, side=30000)
    C = oracle.Colony(xy, 16, seed=seed, keep_pre_ls=1)
    for it in range(1, 16):
        src, _ = C.source()
        C.iterate(12, 1)
        pre, pre_len, checks = C.ant_pre()
        check_construction(xy, C, src, pre, checks, it, seed, 8)
        tours, lens = C.ant_tours()
        D = dmat(xy) if it == 1 else D
        for a in range(len(lens)):
            assert is_perm(tours[a], n)
            assert length(D, tours[a]) == lens[a] <= pre_len[a] == length(D, pre[a])


def test_mmas_special_case_fallbacks_pick_nearest_unvisited():
    # min_new_edges > n: the focused rule never triggers (plain MMAS walk);
    # k = 3, bl = 2 forces backup and global fallbacks.
    n = 150
    xy = inputs.uniform(n, seed=401, side=50000)
    C = oracle.Colony(xy, 3, bl_size=2, min_new_edges=n + 1, keep_pre_ls=1)
    cand, backup, _ = C.lists()
    xy64 = xy.astype(np.int64)
    idx = np.arange(n)
    fallbacks = 0
    for it in range(3):
        C.iterate(6, 1)
        pre, _, _ = C.ant_pre()
        st = C.ant_stats()
        assert (st[:, oracle.ST_ACO_STEPS] == n - 1).all()
        for a in range(pre.shape[0]):
            r = pre[a]
            vis = np.zeros(n, bool)
            vis[r[0]] = True
            for i in range(n - 1):
                u, v = r[i], r[i + 1]
                if (~vis[cand[u]]).any():
                    assert v in cand[u] and not vis[v]
                else:
                    fallbacks += 1
                    m = ((xy64 - xy64[u]) ** 2).sum(1)
                    m = np.where(vis, np.iinfo(np.int64).max, m)
                    assert v == np.lexsort((idx, m))[0]
                vis[v] = True
    assert fallbacks > 50


def convex_polygon(n, R=100000):
    ang = 2 * np.pi * np.arange(n) / n
    pts = np.stack([np.rint(R + R * np.cos(ang)), np.rint(R + R * np.sin(ang))], 1)
    perm = np.random.default_rng(n).permutation(n)  # hide the hull order
    return pts[perm].astype(np.int32), np.argsort(perm).astype(np.int32)


def same_cycle(a, b):
    return edge_set(a) == edge_set(b)


def test_pheromone_decay_and_fixed_point_on_convex_polygon():
    n = 40
    xy, hull = convex_polygon(n)
    C = oracle.Colony(xy, 16)
    assert same_cycle(C.initial()[0], hull)
    cand, _, _ = C.lists()
    lim0 = C.limits()
    tmax, tmin = np.float32(lim0[2]), np.float32(lim0[3])
    assert tmax > 0 and 0 < tmin < tmax
    tau = C.tau()
    assert (tau == tmax).all()
    on_hull = np.zeros(cand.shape, bool)
    E = edge_set(hull)
    for u in range(n):
        for s in range(cand.shape[1]):
            on_hull[u, s] = frozenset((u, int(cand[u, s]))) in E
    for t in range(1, 25):
        hist, _ = C.iterate(8, 1)
        assert same_cycle(C.source()[0], hull) and same_cycle(C.best()[0], hull)
        assert hist[0, 0] == hist[0, 2] == length(dmat(xy), hull) if t == 1 else True
        lim = C.limits()
        assert np.float32(lim[2]) == tmax and np.float32(lim[3]) == tmin  # gb never improves
        tau = C.tau()
        assert (tau[on_hull] == tmax).all()  # rho*tau_max + 1/L = tau_max exactly
        want = max(tmin, np.float32(tmax * np.float32(2.0 ** -t)))
        assert (tau[~on_hull] == want).all()
        # symmetry of the stored entries
        for u in range(0, n, 7):
            for s in range(cand.shape[1]):
                v = cand[u, s]
                back = np.nonzero(cand[v] == u)[0]
                if back.size:
                    assert tau[v, back[0]] == tau[u, s]
    assert (tau[~on_hull] == tmin).all()


def brute_optimum(xy):
    D = dmat(xy)
    n = len(xy)
    best = None
    for perm in itertools.permutations(range(1, n)):
        if perm[0] > perm[-1]:
            continue
        L = D[0, perm[0]] + D[perm[-1], 0] + sum(D[perm[i], perm[i + 1]] for i in range(n - 2))
        best = L if best is None or L < best else best
    return int(best)


@pytest.mark.parametrize("n", [5, 6, 7, 8, 9])
def test_small_instances_reach_the_exhaustive_optimum(n):
    for inst in range(6 if n == 9 else 10):
        xy = inputs.uniform(n, seed=1000 * n + inst, side=1000)
        C = oracle.Colony(xy, 16, seed=inst + 1)
        C.iterate(8, 30)
        assert C.best()[1] == brute_optimum(xy)


def test_limits_follow_global_best():
    xy = inputs.uniform(300, seed=77)
    C = oracle.Colony(xy, 16)
    for _ in range(5):
        hist, _ = C.iterate(16, 1)
        lim = C.limits()
        gb = C.best()[1]
        assert hist[0, 2] == gb
        # tau_max (1 - rho) L_gb = 1 up to one rounding of the double division
        assert abs(lim[0] * 0.5 * gb - 1.0) < 1e-15
        assert lim[2] == np.float32(lim[0]) and lim[3] == np.float32(lim[1])
        assert 0 < lim[1] < lim[0]
        assert (C.tau() >= np.float32(lim[1])).all() and (C.tau() <= np.float32(lim[0])).all()


def test_base_faco_keeps_constructed_tours():
    """Base FACO (no local search on new tours; the study of min_new_edges,
    Figs. 1 and 3): every ant's final tour is its constructed tour, so its
    length is the constructed length; with the same seed and the same
    source, iteration 1's tours are the pre-search tours of FACO+LS; the
    initial tour is the same (its local search is part of the set-up)."""
    xy = inputs.uniform(600, seed=61)
    base = oracle.Colony(xy, 16, local_search=0, keep_pre_ls=1, min_new_edges=40, rho=0.9, threads=4)
    ls = oracle.Colony(xy, 16, local_search=1, keep_pre_ls=1, min_new_edges=40, rho=0.9, threads=4)
    assert base.initial()[1] == ls.initial()[1]
    np.testing.assert_array_equal(base.initial()[0], ls.initial()[0])
    _, base_len = base.iterate(10, 1)
    _, ls_len = ls.iterate(10, 1)
    bt, bl = base.ant_tours()
    pt, pl, _ = base.ant_pre()
    np.testing.assert_array_equal(bt, pt)
    np.testing.assert_array_equal(bl, pl)
    np.testing.assert_array_equal(bl, base_len[0])
    for a in range(10):
        assert bl[a] == oracle.tour_length(xy, bt[a])
        assert sorted(bt[a].tolist()) == list(range(600))
    lpt, lpl, _ = ls.ant_pre()
    np.testing.assert_array_equal(bt, lpt)  # same construction before any search
    assert np.all(ls_len[0] <= base_len[0]) and np.any(ls_len[0] < base_len[0])
    # later iterations: base FACO's tours stay constructed tours
    base.iterate(10, 4)
    bt, bl = base.ant_tours()
    pt, pl, _ = base.ant_pre()
    np.testing.assert_array_equal(bt, pt)


# ---- trail limits (Sec. 4.5) and the source choice (Sec. 5.2) ---------------

@pytest.mark.parametrize("n,k", [(40, 16), (300, 16), (300, 8), (1000, 5), (2500, 32), (700, 2)])
def test_tau_min_meets_its_defining_probability(n, k):
    """Sec. 4.5: tau_min is set so that, once the trails have converged (one
    edge at tau_max among `avg` choices, the rest at tau_min), an ant picking
    by pheromone alone takes the tau_max edge at each of its n decisions with
    probability p_dec = tau_max / (tau_max + (avg - 1) tau_min), and builds
    the best solution with probability p_dec^n = p_best.  FACO with local
    search takes avg = cl_size (the candidate list length k).  The check is
    the derivation's property, not the closed form: a wrong avg (the MMAS
    n/2), a dropped n-th root or a swapped (avg - 1) gives another p_dec^n."""
    xy = inputs.uniform(n, seed=500 + n + k)
    for p_best in (0.05, 0.5):
        C = oracle.Colony(xy, k, p_best=p_best)
        tmax, tmin, tmax32, tmin32 = C.limits()
        kk = min(k, n - 1)
        p_dec = tmax / (tmax + (kk - 1) * tmin)
        # p_dec^n = exp(n log p_dec): relative error ~ n * 1e-16 from rounding
        assert abs(math.exp(n * math.log(p_dec)) / p_best - 1.0) < 1e-11 * n
        # the same colony with another p_best moves tau_min the right way
        assert tmin32 == np.float32(tmin) and tmax32 == np.float32(tmax)
    lo = oracle.Colony(xy, k, p_best=0.01).limits()[1]
    hi = oracle.Colony(xy, k, p_best=0.5).limits()[1]
    assert hi < lo  # a larger p_best means a sharper contrast, a smaller tau_min


def _source_run(xy, p_src, iters, seed=3, ants=3):
    C = oracle.Colony(xy, 16, seed=seed, p_source_gb=p_src, threads=2)
    rows = []
    for it in range(1, iters + 1):
        hist, alh = C.iterate(ants, 1)
        tours, lens = C.ant_tours()
        src, src_len = C.source()
        best, best_len = C.best()
        rows.append((it, hist[0], alh[0], tours, lens, src, src_len, best, best_len))
    return rows


@pytest.mark.parametrize("p_src", [0.01, 0.3])
def test_source_is_global_best_with_probability_p(p_src):
    """Alg 2 ("choose between global_best and iter_best"), Sec. 5.2: after
    each iteration the source is the best-so-far tour with probability
    p_source_gb, else the iteration's best tour (shortest, lowest ant index
    on ties).  Checked iteration by iteration against the tours themselves,
    and the share of global-best sources against a binomial bound; an
    inverted draw (global best with probability 1 - p) fails both."""
    xy = inputs.uniform(30, seed=91, side=3000)
    iters = 600
    rows = _source_run(xy, p_src, iters)
    used_gb = 0
    for it, h, alh, tours, lens, src, src_len, best, best_len in rows:
        ib = int(np.argmin(lens))  # first index of the minimum
        assert h[0] == lens[ib] and h[1] == ib and h[2] == best_len
        np.testing.assert_array_equal(alh, lens)
        if h[3]:
            used_gb += 1
            np.testing.assert_array_equal(src, best)
            assert src_len == best_len
        else:
            np.testing.assert_array_equal(src, tours[ib])
            assert src_len == lens[ib]
        # the decision is the colony's Philox draw (tag 1, draw 0) of this
        # iteration; the generator itself is pinned by known-answer vectors
        assert bool(h[3]) == (oracle.u01(oracle.draw(3, 0, 0, it, 1)) < p_src)
    mean, sd = iters * p_src, math.sqrt(iters * p_src * (1 - p_src))
    assert abs(used_gb - mean) <= 5 * sd + 1
    # the two arms must both occur for the check above to mean anything
    assert 0 < used_gb < iters


@pytest.mark.parametrize("p_src,want", [(0.0, 0), (1.0, 1)])
def test_source_choice_extremes(p_src, want):
    """p_source_gb = 0: always the iteration best; = 1: always the best so
    far (u01 < 1 always holds)."""
    rows = _source_run(inputs.uniform(25, seed=92, side=3000), p_src, 40)
    for it, h, alh, tours, lens, src, src_len, best, best_len in rows:
        assert h[3] == want
        np.testing.assert_array_equal(src, best if want else tours[int(np.argmin(lens))])


# ---- the initial tour's 3-opt segment exchange (Sec. 4.3) --------------------

def best_exchange_delta(D, route, min_seg=2):
    """Smallest length change over every exchange of two adjacent tour
    sections (X Y Z -> X Z Y, no reversal) whose three sections each hold
    at least `min_seg` nodes, by explicit tour surgery."""
    n = len(route)
    L0 = length(D, route)
    best = 0
    r = list(route)
    for i in range(n):
        rot = r[i:] + r[:i]  # X starts at position 0
        for j in range(min_seg, n):  # X = rot[:j]
            for k in range(j + min_seg, n - min_seg + 1):  # Y = rot[j:k], Z = rot[k:]
                t = rot[:j] + rot[k:] + rot[j:k]
                best = min(best, length(D, t) - L0)
    return best


@pytest.mark.parametrize("seed", range(6))
def test_three_opt_search_reaches_exchange_optimum(seed):
    """With full neighbour lists, the local search with the segment exchange
    ends in a tour that no 2-opt move, no Or-opt move and no exchange of two
    adjacent sections (each section of >= 2 nodes) improves, checked by
    exhaustive tour surgery; the returned gain is the length difference."""
    n = 16 + 2 * seed
    xy = inputs.uniform(n, seed=700 + seed, side=10000)
    D = dmat(xy)
    cand = oracle.knn_rows(xy, n - 1)
    route = oracle.nn_tour(xy, cand[:, :3], cand[:, 3:6])
    L0 = length(D, route)
    out, gain, st = oracle.local_search(xy, cand, route, route.copy(), oropt=1, verify=1, three_opt=1)
    assert st[oracle.ST_MOVES_2OPT] + st[oracle.ST_MOVES_OR] + st[oracle.ST_MOVES_3OPT] < n
    assert is_perm(out, n)
    assert length(D, out) == L0 - gain
    assert best_2opt_delta(D, list(out)) == 0
    assert best_oropt_delta(D, list(out)) == 0
    assert best_exchange_delta(D, list(out)) == 0


def test_three_opt_moves_occur_and_only_shorten():
    """On 2-opt + Or-opt local optima of larger instances the exchange still
    finds moves; each search only shortens the tour, and without the flag
    the search is the plain one."""
    found = 0
    for seed in range(8):
        n = 60
        xy = inputs.uniform(n, seed=800 + seed, side=10000)
        D = dmat(xy)
        cand = oracle.knn_rows(xy, 8)
        route = oracle.nn_tour(xy, cand[:, :3], cand[:, 3:6])
        base, g0, _ = oracle.local_search(xy, cand, route, route.copy(), oropt=1, verify=1, three_opt=0)
        plain, gp, _ = oracle.local_search(xy, cand, route, route.copy(), oropt=1, verify=1)
        np.testing.assert_array_equal(base, plain)
        assert g0 == gp
        out, g1, st = oracle.local_search(xy, cand, base, base.copy(), oropt=1, verify=1, three_opt=1)
        assert is_perm(out, n) and g1 >= 0
        assert length(D, out) == length(D, base) - g1
        found += int(st[oracle.ST_MOVES_3OPT])
    assert found > 0


def test_initial_tour_with_three_opt():
    """The colony's initial tour with init_3opt: a permutation whose length
    is the recomputed one (the search takes another path than without the
    flag, so neither local optimum bounds the other), and exchange-optimal
    for full neighbour lists on a small instance."""
    moved = 0
    for n, seed in ((300, 3), (500, 4)):
        xy = inputs.uniform(n, seed=seed)
        a = oracle.Colony(xy, 16)
        b = oracle.Colony(xy, 16, init_3opt=1)
        ra, La = a.initial()
        rb, Lb = b.initial()
        assert is_perm(rb, n) and Lb == oracle.tour_length(xy, rb)
        moved += int(La != Lb)
    assert moved > 0
    xy = inputs.uniform(22, seed=41, side=5000)
    c = oracle.Colony(xy, 21, init_3opt=1, bl_size=0)
    r, L = c.initial()
    D = dmat(xy)
    assert best_2opt_delta(D, list(r)) == 0 and best_exchange_delta(D, list(r)) == 0
