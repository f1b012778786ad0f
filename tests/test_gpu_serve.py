"""The request server (include/faco_serve.h) on a GB300: every request's
result equals the one-colony path with its seed, alone and in a mix of
uneven requests; admission waits for device memory; mixed list widths.
"""
import numpy as np
import pytest

from paper_2203_02228_gb300 import Colony, FacoError, Server, inputs, _lib

pytestmark = pytest.mark.gpu


def plain(xy, k, ants, budget, seed, **kw):
    c = Colony(xy, k, seed=seed, **kw)
    c.iterate(ants, budget)
    t, L = c.best()
    c.close()
    return t, L


def test_result_alone_equals_result_in_the_mix():
    target = inputs.stippled(700, seed=77, blobs=5, ridges=1, side=40_000)
    want = plain(target, 16, 24, 12, 5)
    with Server(2 << 30) as s:
        t = s.submit(target, 16, 24, 12, 5)
        alone = s.wait(t)
        s.release(t)
        # the same request again, between uneven others that overlap it
        others = []
        for j, n in enumerate([2500, 300, 1200, 9000, 450, 60]):
            xy = inputs.uniform(n, seed=300 + j)
            others.append((xy, s.submit(xy, 16, 8 + 8 * (j % 3), 5 + 4 * j, 100 + j), 8 + 8 * (j % 3),
                           5 + 4 * j, 100 + j))
            if j == 2:
                t2 = s.submit(target, 16, 24, 12, 5)
        mixed = s.wait(t2)
        for xy, tk, ants, budget, seed in others:
            got = s.wait(tk)
            ref = plain(xy, 16, ants, budget, seed)
            assert got[1] == ref[1]
            np.testing.assert_array_equal(got[0], ref[0])
        st = s.stats()
    assert alone[1] == mixed[1] == want[1]
    np.testing.assert_array_equal(alone[0], want[0])
    np.testing.assert_array_equal(mixed[0], want[0])
    assert alone[3] >= alone[2] and mixed[3] >= mixed[2]
    assert st["completed"] == 8 and st["peak_active"] >= 2 and st["pool_in_use"] == 0


def test_admission_waits_for_memory():
    xs = [inputs.uniform(n, seed=900 + n) for n in (1500, 1700, 1600, 1400, 1550)]
    with Server(1 << 30) as probe:
        need = max(probe.request_bytes(x.shape[0], 16, 32) for x in xs)
    pool = int(need * 2.5)  # room for two at a time
    with Server(pool) as s:
        tickets = [s.submit(x, 16, 32, 6, 40 + i) for i, x in enumerate(xs)]
        res = [s.wait(t) for t in tickets]
        st = s.stats()
        too_big = inputs.uniform(3000, seed=5)
        with pytest.raises(FacoError):
            s.submit(too_big, 16, 512, 1, 1)
    assert st["peak_active"] <= 2
    for i, x in enumerate(xs):
        ref = plain(x, 16, 32, 6, 40 + i)
        assert res[i][1] == ref[1]
        np.testing.assert_array_equal(res[i][0], ref[0])


def test_mixed_list_widths_and_parameters():
    xs = [inputs.uniform(n, seed=n) for n in (400, 800, 1300)]
    with Server(1 << 30, rho=0.9, min_new_edges=12) as s:
        t16 = s.submit(xs[0], 16, 16, 7, 3)
        t24 = s.submit(xs[1], 24, 16, 5, 4)
        t8 = s.submit(xs[2], 8, 16, 9, 5)
        r16, r24, r8 = s.wait(t16), s.wait(t24), s.wait(t8)
        assert s.poll(t16) is not None
        s.release(t16)
        with pytest.raises(FacoError):
            s.poll(t16)
    for (xy, k, b, seed), r in zip([(xs[0], 16, 7, 3), (xs[1], 24, 5, 4), (xs[2], 8, 9, 5)], [r16, r24, r8]):
        ref = plain(xy, k, 16, b, seed, rho=0.9, min_new_edges=12)
        assert r[1] == ref[1]
        np.testing.assert_array_equal(r[0], ref[0])


def test_submit_rejects_bad_requests():
    with Server(64 << 20) as s:
        xy = inputs.uniform(100, seed=1)
        L = s._L
        T = _lib.ctypes.c_uint64()
        P = xy.ctypes.data_as(_lib.ctypes.c_void_p)
        assert L.faco_server_submit(s._h, P, 2, 16, 4, 1, 1, _lib.ctypes.byref(T)) == _lib.FACO_E_ARG
        assert L.faco_server_submit(s._h, P, 100, 16, 0, 1, 1, _lib.ctypes.byref(T)) == _lib.FACO_E_ARG
        assert L.faco_server_submit(s._h, P, 100, 16, 4, 0, 1, _lib.ctypes.byref(T)) == _lib.FACO_E_ARG
        assert L.faco_server_submit(s._h, P, 300000, 16, 4, 1, 1, _lib.ctypes.byref(T)) == _lib.FACO_E_SIZE
        bad = xy.copy()
        bad[7, 1] = -3
        assert L.faco_server_submit(s._h, bad.ctypes.data_as(_lib.ctypes.c_void_p), 100, 16, 4, 1, 1,
                                    _lib.ctypes.byref(T)) == _lib.FACO_E_ARG
        big = inputs.uniform(50000, seed=2)
        with pytest.raises(FacoError):
            s.submit(big, 16, 256, 1, 1)  # can never fit 64 MB


def test_served_results_equal_the_oracle():
    """Requests served in a mix give the oracle's tours and lengths (Alg 2
    with the request's seed) -- checked against the CPU statement of the
    method, not only against the one-colony GPU path."""
    import oracle

    reqs = [(inputs.stippled(900, seed=81, blobs=6, ridges=1, side=50_000), 16, 8, 21),
            (inputs.uniform(1500, seed=82), 24, 10, 22),
            (inputs.uniform(420, seed=83), 16, 6, 23),
            (inputs.uniform(2600, seed=84), 16, 4, 24)]
    with Server(2 << 30) as s:
        tickets = [s.submit(xy, 16, ants, budget, seed) for xy, ants, budget, seed in reqs]
        got = [s.wait(t) for t in tickets]
        st = s.stats()
    assert st["peak_active"] >= 2
    for (xy, ants, budget, seed), g in zip(reqs, got):
        o = oracle.Colony(xy, 16, seed=seed, threads=8)
        o.iterate(ants, budget)
        tour, L = o.best()
        assert g[1] == L
        np.testing.assert_array_equal(g[0], tour)
