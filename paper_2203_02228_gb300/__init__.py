"""GB300-native Focused ACO (Skinderowicz, Applied Soft Computing 2022).

Python face of libfaco.so (C ABI in include/faco.h).  The functions keep the
C names (faco_create, faco_iterate, faco_best, ...); ``Colony`` bundles them
for one instance.  PyTorch is only used, when given, for the CUDA stream and
for device-resident input/output buffers.

    from paper_2203_02228_gb300 import Colony, inputs
    col = Colony(inputs.uniform(1000), k=16)
    col.iterate(ants=32, budget=200)
    tour, length = col.best()
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import FacoError, faco_params, faco_stats, load, params_default  # noqa: F401

__all__ = ["Batch", "Colony", "FacoError", "Server", "faco_params", "faco_stats", "load", "params_default",
           "faco_create", "faco_create_ex", "faco_create_device", "faco_iterate", "faco_sync",
           "faco_best", "faco_best_device", "faco_stats_get", "faco_destroy", "faco_strerror"]


def _ptr(a) -> ctypes.c_void_p:
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


# ---- C ABI, same names ---------------------------------------------------

def faco_create(coords_xy: np.ndarray, n: int, k: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _lib.check(load().faco_create(_ptr(coords_xy), n, k, ctypes.byref(h)), "faco_create")
    return h


def faco_create_ex(coords_xy: np.ndarray, n: int, k: int, params: faco_params | None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    p = ctypes.byref(params) if params is not None else None
    _lib.check(load().faco_create_ex(_ptr(coords_xy), n, k, p, ctypes.byref(h)), "faco_create_ex")
    return h


def faco_create_device(coords_xy_dev, n: int, k: int, params: faco_params | None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    p = ctypes.byref(params) if params is not None else None
    _lib.check(load().faco_create_device(_ptr(coords_xy_dev), n, k, p, ctypes.byref(h)), "faco_create_device")
    return h


def faco_iterate(h, ants: int, budget: int) -> None:
    _lib.check(load().faco_iterate(h, ants, budget), "faco_iterate")


def faco_sync(h) -> None:
    _lib.check(load().faco_sync(h), "faco_sync")


def faco_best(h, tour: np.ndarray | None, length: int) -> int:
    L = ctypes.c_int64()
    _lib.check(load().faco_best(h, _ptr(tour), length, ctypes.byref(L)), "faco_best")
    return int(L.value)


def faco_best_device(h, tour_dev, length_dev) -> None:
    _lib.check(load().faco_best_device(h, _ptr(tour_dev), _ptr(length_dev)), "faco_best_device")


def faco_stats_get(h) -> faco_stats:
    s = faco_stats()
    _lib.check(load().faco_stats_get(h, ctypes.byref(s)), "faco_stats_get")
    return s


def faco_destroy(h) -> None:
    load().faco_destroy(h)


def faco_strerror(status: int) -> str:
    return _lib.strerror(status)


# ---- convenience wrapper -------------------------------------------------

class Colony:
    """One FACO colony on the GPU (all state resident on the device)."""

    def __init__(self, coords, k: int = 16, params: faco_params | None = None, device: bool = False,
                 stream=None, **kw):
        p = params if params is not None else params_default()
        for key, v in kw.items():
            setattr(p, key, v)
        if stream is not None:
            p.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.params = p
        self._L = load()
        if device:
            n = int(coords.shape[0])
            self._h = faco_create_device(coords, n, k, p)
        else:
            coords = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 2)
            n = coords.shape[0]
            self._h = faco_create_ex(coords, n, k, p)
        st = self.stats()
        self.n, self.k, self.bl = st.n, st.k, st.bl

    def close(self) -> None:
        if getattr(self, "_h", None):
            faco_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def handle(self):
        return self._h

    def iterate(self, ants: int, budget: int = 1) -> None:
        faco_iterate(self._h, ants, budget)

    def sync(self) -> None:
        faco_sync(self._h)

    def best(self):
        tour = np.zeros(self.n, np.int32)
        L = faco_best(self._h, tour, self.n)
        return tour, L

    def best_device(self, tour_dev, length_dev) -> None:
        faco_best_device(self._h, tour_dev, length_dev)

    def stats(self) -> faco_stats:
        return faco_stats_get(self._h)

    def lists(self):
        cand = np.zeros((self.n, self.k), np.int32)
        backup = np.zeros((self.n, max(self.bl, 1)), np.int32)
        eta = np.zeros((self.n, self.k), np.float32)
        _lib.check(self._L.faco_get_lists(self._h, _ptr(cand), _ptr(backup), _ptr(eta)), "faco_get_lists")
        return cand, backup[:, :self.bl], eta

    def tau(self) -> np.ndarray:
        t = np.zeros((self.n, self.k), np.float32)
        _lib.check(self._L.faco_get_tau(self._h, _ptr(t)), "faco_get_tau")
        return t

    def limits(self) -> np.ndarray:
        out = np.zeros(4, np.float64)
        _lib.check(self._L.faco_get_limits(self._h, _ptr(out)), "faco_get_limits")
        return out

    def _route(self, fn, what):
        r = np.zeros(self.n, np.int32)
        L = ctypes.c_int64()
        _lib.check(fn(self._h, _ptr(r), ctypes.byref(L)), what)
        return r, int(L.value)

    def source(self):
        return self._route(self._L.faco_get_source, "faco_get_source")

    def initial(self):
        return self._route(self._L.faco_get_initial, "faco_get_initial")

    def history(self, max_iters: int = 1 << 20) -> np.ndarray:
        st = self.stats()
        m = min(max_iters, st.iteration)
        h = np.zeros((max(m, 1), 4), np.int64)
        rows = ctypes.c_int64()
        _lib.check(self._L.faco_get_history(self._h, _ptr(h), m, ctypes.byref(rows)), "faco_get_history")
        return h[:rows.value]

    def ant_stats(self) -> np.ndarray:
        m = self.stats().ants
        st = np.zeros((m, 24), np.int64)
        _lib.check(self._L.faco_get_ant_stats(self._h, _ptr(st)), "faco_get_ant_stats")
        return st

    def profile(self, on: bool = True) -> None:
        _lib.check(self._L.faco_profile_enable(self._h, int(on)), "faco_profile_enable")

    def profile_read(self):
        ms = ctypes.c_double()
        cnt = ctypes.c_int64()
        _lib.check(self._L.faco_profile_read(self._h, ctypes.byref(ms), ctypes.byref(cnt)), "faco_profile_read")
        return float(ms.value), int(cnt.value)

    def ant_tours(self):
        m = self.stats().ants
        t = np.zeros((m, self.n), np.int32)
        lens = np.zeros(m, np.int64)
        _lib.check(self._L.faco_get_ant_tours(self._h, _ptr(t), _ptr(lens)), "faco_get_ant_tours")
        return t, lens

    def ant_pre(self):
        m = self.stats().ants
        t = np.zeros((m, self.n), np.int32)
        lens = np.zeros(m, np.int64)
        chk = np.zeros((m, self.n), np.int32)
        nchk = np.zeros(m, np.int32)
        _lib.check(self._L.faco_get_ant_pre(self._h, _ptr(t), _ptr(lens), _ptr(chk), _ptr(nchk)),
                   "faco_get_ant_pre")
        return t, lens, [chk[i, :nchk[i]].copy() for i in range(m)]


class Batch:
    """Independent colonies run through the same launches (include/faco_batch.h).

    Colony i equals ``Colony(coords[i], k, params with seed=seeds[i])`` driven by
    the same ``iterate`` calls, bit for bit; the batch only shares the GPU.
    """

    def __init__(self, coords_list, k: int = 16, params: faco_params | None = None, seeds=None,
                 stream=None, plan: int | None = None, **kw):
        p = params if params is not None else params_default()
        for key, v in kw.items():
            setattr(p, key, v)
        if stream is not None:
            p.stream = ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        self.params = p
        self._L = load()
        self._coords = [np.ascontiguousarray(c, dtype=np.int32).reshape(-1, 2) for c in coords_list]
        self.count = len(self._coords)
        self.ns = np.array([c.shape[0] for c in self._coords], dtype=np.int32)
        ptrs = (ctypes.c_void_p * self.count)(*[c.ctypes.data for c in self._coords])
        sd = None
        if seeds is not None:
            self._seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
            assert self._seeds.shape[0] == self.count
            sd = self._seeds.ctypes.data_as(ctypes.c_void_p)
        h = ctypes.c_void_p()
        _lib.check(self._L.faco_batch_create(ctypes.cast(ptrs, ctypes.c_void_p), _ptr(self.ns), self.count, k,
                                             ctypes.byref(p), sd, ctypes.byref(h)), "faco_batch_create")
        self._h = h
        self._coords = None  # copied by the library
        if plan is not None:
            self.set_plan(plan)

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.faco_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def iterate(self, ants: int, budget: int = 1) -> None:
        _lib.check(self._L.faco_batch_iterate(self._h, ants, budget), "faco_batch_iterate")

    def sync(self) -> None:
        _lib.check(self._L.faco_batch_sync(self._h), "faco_batch_sync")

    def best(self, i: int):
        tour = np.empty(int(self.ns[i]), np.int32)
        L = ctypes.c_int64()
        _lib.check(self._L.faco_batch_best(self._h, i, _ptr(tour), tour.shape[0], ctypes.byref(L)),
                   "faco_batch_best")
        return tour, int(L.value)

    def tours(self):
        """All global-best tours (list of arrays) and lengths."""
        flat = np.empty(int(self.ns.sum()), np.int32)
        lens = np.empty(self.count, np.int64)
        _lib.check(self._L.faco_batch_tours(self._h, _ptr(flat), _ptr(lens)), "faco_batch_tours")
        off = np.concatenate([[0], np.cumsum(self.ns)])
        return [flat[off[i]:off[i + 1]] for i in range(self.count)], lens

    def lengths(self) -> np.ndarray:
        lens = np.empty(self.count, np.int64)
        _lib.check(self._L.faco_batch_tours(self._h, None, _ptr(lens)), "faco_batch_tours")
        return lens

    def stats(self, i: int) -> faco_stats:
        s = faco_stats()
        _lib.check(self._L.faco_batch_stats(self._h, i, ctypes.byref(s)), "faco_batch_stats")
        return s

    def tau(self, i: int) -> np.ndarray:
        st = self.stats(i)
        t = np.empty((st.n, st.k), np.float32)
        _lib.check(self._L.faco_batch_tau(self._h, i, _ptr(t)), "faco_batch_tau")
        return t

    def set_plan(self, mode: int) -> None:
        _lib.check(self._L.faco_batch_set_plan(self._h, mode), "faco_batch_set_plan")

    def plan(self) -> np.ndarray:
        v = np.empty(self.count, np.int32)
        _lib.check(self._L.faco_batch_get_plan(self._h, _ptr(v)), "faco_batch_get_plan")
        return v


class Server:
    """Request server (include/faco_serve.h): instances admitted by device
    memory, set up while others iterate, iterated in rounds shared with the
    requests of their cohort (roulette width and size class).

    A request's tour and length equal those of a Colony with the server's
    parameters and the request's seed, alone or in any mix.
    """

    def __init__(self, device_bytes: int, params: faco_params | None = None, **kw):
        p = params if params is not None else params_default()
        for key, v in kw.items():
            setattr(p, key, v)
        self.params = p
        self._L = load()
        h = ctypes.c_void_p()
        _lib.check(self._L.faco_server_create(int(device_bytes), ctypes.byref(p), ctypes.byref(h)),
                   "faco_server_create")
        self._h = h
        self._n = {}

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._L.faco_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def request_bytes(self, n: int, k: int, ants: int) -> int:
        return int(self._L.faco_server_request_bytes(n, k, ants, ctypes.byref(self.params)))

    def submit(self, coords, k: int, ants: int, budget: int, seed: int) -> int:
        xy = np.ascontiguousarray(coords, dtype=np.int32).reshape(-1, 2)
        t = ctypes.c_uint64()
        _lib.check(self._L.faco_server_submit(self._h, _ptr(xy), xy.shape[0], k, ants, budget, seed,
                                              ctypes.byref(t)), "faco_server_submit")
        self._n[t.value] = xy.shape[0]
        return int(t.value)

    def poll(self, ticket: int):
        """None while pending, else (tour, length, t_submit_ns, t_done_ns)."""
        n = self._n.get(ticket, 0)  # unknown tickets: the library reports FACO_E_ARG
        tour = np.empty(n, np.int32)
        L, ts, td = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        rc = self._L.faco_server_poll(self._h, ticket, _ptr(tour), n, ctypes.byref(L), ctypes.byref(ts),
                                      ctypes.byref(td))
        if rc == _lib.FACO_PENDING:
            return None
        _lib.check(rc, "faco_server_poll")
        return tour, int(L.value), int(ts.value), int(td.value)

    def wait(self, ticket: int, timeout_ms: int = 600_000):
        rc = self._L.faco_server_wait(self._h, ticket, timeout_ms)
        if rc == _lib.FACO_PENDING:
            raise TimeoutError("request %d still pending after %d ms" % (ticket, timeout_ms))
        return self.poll(ticket)

    def release(self, ticket: int) -> None:
        _lib.check(self._L.faco_server_release(self._h, ticket), "faco_server_release")
        self._n.pop(ticket, None)

    def stats(self):
        st = _lib.faco_server_stats()
        _lib.check(self._L.faco_server_stats_get(self._h, ctypes.byref(st)), "faco_server_stats_get")
        return {f: getattr(st, f) for f, _ in st._fields_}


def tuner_report(max_rows: int = 256) -> list:
    """The batch/server kernel tuner's timings on the current device (see
    faco_batch_tuner_report): one dict per tuned size class."""
    rows = np.zeros((max_rows, 9), np.float64)
    cnt = ctypes.c_int32()
    _lib.check(load().faco_batch_tuner_report(_ptr(rows), max_rows, ctypes.byref(cnt)), "faco_batch_tuner_report")
    names = ("segment_table", "arrays_2_blocks_per_sm", "arrays_4_blocks_per_sm", "arrays_8_blocks_per_sm")
    out = []
    for r in rows[:min(cnt.value, max_rows)]:
        c = int(r[0])
        out.append({"size_class": c, "n_range": [0 if c == 0 else 512 * 4 ** (c - 1), 512 * 4 ** c - 1],
                    "ants": int(r[1]), "roulette_width": int(r[2]), "goal": ("batch", "latency")[int(r[3])],
                    "chosen": names[int(r[4])] if r[4] >= 0 else None,
                    "ms": {nm: (float(v) if v >= 0 else None) for nm, v in zip(names, r[5:9])}})
    return out


def l2_probe(bytes_: int = 48 << 20, reps: int = 200) -> float:
    """L2 read bandwidth of the current device in GB/s (see faco_l2_probe)."""
    g = ctypes.c_double()
    _lib.check(load().faco_l2_probe(int(bytes_), int(reps), ctypes.byref(g)), "faco_l2_probe")
    return float(g.value)


def device_selftest(what: int, inp: np.ndarray, out: np.ndarray, count: int, width: int = 16, seed: int = 0) -> None:
    """Runs a device primitive through the library (see faco_test_device)."""
    _lib.check(load().faco_test_device(what, _ptr(inp), inp.nbytes, _ptr(out), out.nbytes, count, width, seed),
               "faco_test_device")


def pool_replay(pool_bytes: int, ops: np.ndarray) -> np.ndarray:
    """Replays take / give-back operations on the server's device-memory
    allocator, on the host (see faco_test_pool).  ops: int64 [count][2];
    returns int64 [count][2] (offset taken or -1, bytes in use after)."""
    ops = np.ascontiguousarray(ops, dtype=np.int64)
    out = np.zeros_like(ops)
    _lib.check(load().faco_test_pool(int(pool_bytes), _ptr(ops), int(ops.shape[0]), _ptr(out)), "faco_test_pool")
    return out
