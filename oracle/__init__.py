"""Plain CPU oracle for Focused ACO -- test infrastructure only.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does; it
shares no code with the oracle.

The C source (``faco_oracle.c``) states every step with the paper section,
equation or algorithm it follows; this module only marshals arguments.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "faco_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

NSTATS = 16
ST_ACO_STEPS, ST_NEW_EDGES, ST_BACKUP, ST_GLOBAL, ST_CHECKLIST, ST_POPS = 0, 1, 2, 3, 4, 5
ST_MOVES_2OPT, ST_MOVES_OR, ST_FLIP_ELEMS, ST_VERIFY_ROUNDS, ST_MOVES_3OPT = 6, 7, 8, 9, 10


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FP contraction, OpenMP over ants)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC),
                                                   os.path.getmtime(os.path.join(_HERE, "faco_oracle.h")))):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("rho", ctypes.c_float),
        ("min_new_edges", ctypes.c_int32),
        ("bl_size", ctypes.c_int32),
        ("p_best", ctypes.c_double),
        ("p_source_gb", ctypes.c_double),
        ("oropt", ctypes.c_int32),
        ("verify_pass", ctypes.c_int32),
        ("threads", ctypes.c_int32),
        ("keep_pre_ls", ctypes.c_int32),
        ("local_search", ctypes.c_int32),
        ("init_3opt", ctypes.c_int32),
    ]


def _P(dt):
    return np.ctypeslib.ndpointer(dtype=dt, flags="C_CONTIGUOUS")


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            vp = ctypes.c_void_p
            L.orc_isqrt.restype = ctypes.c_uint64
            L.orc_isqrt.argtypes = [ctypes.c_uint64]
            L.orc_euc2d.restype = ctypes.c_int32
            L.orc_euc2d.argtypes = [_P(np.int32), ctypes.c_int32, ctypes.c_int32]
            L.orc_philox4x32_10.argtypes = [_P(np.uint32), _P(np.uint32), _P(np.uint32)]
            L.orc_draw.restype = ctypes.c_uint32
            L.orc_draw.argtypes = [ctypes.c_uint64] + [ctypes.c_uint32] * 4
            L.orc_u01.restype = ctypes.c_float
            L.orc_u01.argtypes = [ctypes.c_uint32]
            L.orc_params_default.argtypes = [ctypes.POINTER(Params)]
            L.orc_knn_rows.argtypes = [_P(np.int32), ctypes.c_int32, ctypes.c_int32, _P(np.int32),
                                       ctypes.c_int32, ctypes.c_int32, _P(np.int32)]
            L.orc_roulette.restype = ctypes.c_int32
            L.orc_roulette.argtypes = [_P(np.float32), ctypes.c_int32, ctypes.c_float]
            L.orc_local_search.restype = ctypes.c_int64
            L.orc_local_search.argtypes = [_P(np.int32), ctypes.c_int32, _P(np.int32), ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_int32, _P(np.int32), _P(np.int32),
                                           _P(np.int32), ctypes.c_int32, vp]
            L.orc_local_search_ex.restype = ctypes.c_int64
            L.orc_local_search_ex.argtypes = [_P(np.int32), ctypes.c_int32, _P(np.int32), ctypes.c_int32,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _P(np.int32),
                                              _P(np.int32), _P(np.int32), ctypes.c_int32, vp]
            L.orc_nn_tour.argtypes = [_P(np.int32), ctypes.c_int32, _P(np.int32), ctypes.c_int32,
                                      _P(np.int32), ctypes.c_int32, _P(np.int32)]
            L.orc_tour_length.restype = ctypes.c_int64
            L.orc_tour_length.argtypes = [_P(np.int32), ctypes.c_int32, _P(np.int32)]
            L.orc_create.restype = ctypes.c_int
            L.orc_create.argtypes = [_P(np.int32), ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(Params), ctypes.POINTER(vp)]
            L.orc_destroy.argtypes = [vp]
            L.orc_iterate.restype = ctypes.c_int
            L.orc_iterate.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, vp]
            for name in ("orc_n", "orc_k", "orc_bl", "orc_last_ants"):
                getattr(L, name).restype = ctypes.c_int32
                getattr(L, name).argtypes = [vp]
            L.orc_iteration.restype = ctypes.c_int64
            L.orc_iteration.argtypes = [vp]
            L.orc_get_lists.argtypes = [vp, vp, vp, vp]
            L.orc_get_tau.argtypes = [vp, _P(np.float32)]
            L.orc_get_limits.argtypes = [vp, _P(np.float64)]
            for name in ("orc_get_source", "orc_get_best", "orc_get_initial"):
                getattr(L, name).restype = ctypes.c_int64
                getattr(L, name).argtypes = [vp, vp]
            L.orc_get_ant_tours.argtypes = [vp, vp, vp]
            L.orc_get_ant_stats.argtypes = [vp, _P(np.int64)]
            L.orc_get_ant_pre.restype = ctypes.c_int
            L.orc_get_ant_pre.argtypes = [vp, vp, vp, vp, vp]
            L.orc_set_state.restype = ctypes.c_int
            L.orc_set_state.argtypes = [vp, vp, vp]
            L.orc_set_threads.restype = ctypes.c_int
            L.orc_set_threads.argtypes = [vp, ctypes.c_int32]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_params_default(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


# ---- primitives ----------------------------------------------------------

def isqrt(m: int) -> int:
    return int(lib().orc_isqrt(m))


def euc2d(xy: np.ndarray, a: int, b: int) -> int:
    return int(lib().orc_euc2d(np.ascontiguousarray(xy, dtype=np.int32).reshape(-1), a, b))


def philox(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def draw(seed: int, idx: int, ant: int, it: int, tag: int) -> int:
    return int(lib().orc_draw(seed, idx, ant, it, tag))


def u01(x: int) -> float:
    return float(lib().orc_u01(x))


def roulette(w, u: float) -> int:
    w = np.asarray(w, np.float32)
    width = 16 if len(w) <= 16 else 32
    pad = np.zeros(width, np.float32)
    pad[:len(w)] = w
    return int(lib().orc_roulette(pad, width, ctypes.c_float(u)))


def knn_rows(xy: np.ndarray, K: int, rows=None, threads: int = 0) -> np.ndarray:
    xy = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1)
    n = xy.size // 2
    rows = np.arange(n, dtype=np.int32) if rows is None else np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((rows.size, K), np.int32)
    lib().orc_knn_rows(xy, n, K, rows, rows.size, threads or (os.cpu_count() or 1), out)
    return out


def nn_tour(xy, cand, backup) -> np.ndarray:
    xy = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    backup = np.ascontiguousarray(backup, dtype=np.int32)
    n = xy.size // 2
    out = np.zeros(n, np.int32)
    bl = backup.shape[1] if backup.ndim == 2 and backup.size else 0
    lib().orc_nn_tour(xy, n, cand, cand.shape[1], backup if bl else np.zeros((n, 1), np.int32), bl, out)
    return out


def tour_length(xy: np.ndarray, route: np.ndarray) -> int:
    xy = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1)
    route = np.ascontiguousarray(route, dtype=np.int32)
    return int(lib().orc_tour_length(xy, route.size, route))


def local_search(xy, cand, route, queue, oropt=1, verify=1, three_opt=0):
    """Runs Alg 3 (+ options) on a copy of `route`; returns (route, gain, stats)."""
    xy = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    n = xy.size // 2
    route = np.array(route, dtype=np.int32)
    pos = np.empty(n, np.int32)
    pos[route] = np.arange(n, dtype=np.int32)
    queue = np.ascontiguousarray(queue, dtype=np.int32)
    st = np.zeros(NSTATS, np.int64)
    g = lib().orc_local_search_ex(xy, n, cand, cand.shape[1], oropt, verify, three_opt, route, pos, queue,
                                  queue.size, _ptr(st))
    return route, int(g), st


# ---- colony --------------------------------------------------------------

class Colony:
    """One FACO colony run by the oracle (Alg 2)."""

    def __init__(self, xy: np.ndarray, k: int = 16, params: Params | None = None, **kw):
        self._L = lib()
        self.xy = np.ascontiguousarray(xy, dtype=np.int32).reshape(-1, 2)
        p = params if params is not None else default_params(**kw)
        if params is not None:
            for key, v in kw.items():
                setattr(p, key, v)
        self.params = p
        h = ctypes.c_void_p()
        rc = self._L.orc_create(self.xy.reshape(-1), self.xy.shape[0], k, ctypes.byref(p), ctypes.byref(h))
        if rc != 0:
            raise ValueError("orc_create failed: %d" % rc)
        self._h = h
        self.n = self._L.orc_n(h)
        self.k = self._L.orc_k(h)
        self.bl = self._L.orc_bl(h)

    def close(self):
        if getattr(self, "_h", None):
            self._L.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def iterate(self, ants: int, iters: int):
        hist = np.zeros((iters, 4), np.int64)
        alh = np.zeros((iters, ants), np.int64)
        rc = self._L.orc_iterate(self._h, ants, iters, _ptr(hist), _ptr(alh))
        if rc != 0:
            raise ValueError("orc_iterate failed: %d" % rc)
        return hist, alh

    @property
    def iteration(self) -> int:
        return int(self._L.orc_iteration(self._h))

    def lists(self):
        cand = np.zeros((self.n, self.k), np.int32)
        backup = np.zeros((self.n, max(self.bl, 1)), np.int32)
        eta = np.zeros((self.n, self.k), np.float32)
        self._L.orc_get_lists(self._h, _ptr(cand), _ptr(backup), _ptr(eta))
        return cand, backup[:, :self.bl], eta

    def tau(self) -> np.ndarray:
        t = np.zeros((self.n, self.k), np.float32)
        self._L.orc_get_tau(self._h, t)
        return t

    def limits(self):
        out = np.zeros(4, np.float64)
        self._L.orc_get_limits(self._h, out)
        return out

    def _route(self, fn):
        r = np.zeros(self.n, np.int32)
        L = fn(self._h, _ptr(r))
        return r, int(L)

    def source(self):
        return self._route(self._L.orc_get_source)

    def best(self):
        return self._route(self._L.orc_get_best)

    def initial(self):
        return self._route(self._L.orc_get_initial)

    def ant_tours(self):
        m = self._L.orc_last_ants(self._h)
        t = np.zeros((m, self.n), np.int32)
        lens = np.zeros(m, np.int64)
        self._L.orc_get_ant_tours(self._h, _ptr(t), _ptr(lens))
        return t, lens

    def ant_stats(self):
        m = self._L.orc_last_ants(self._h)
        st = np.zeros((m, NSTATS), np.int64)
        self._L.orc_get_ant_stats(self._h, st)
        return st

    def ant_pre(self):
        m = self._L.orc_last_ants(self._h)
        t = np.zeros((m, self.n), np.int32)
        lens = np.zeros(m, np.int64)
        chk = np.zeros((m, self.n), np.int32)
        nchk = np.zeros(m, np.int32)
        rc = self._L.orc_get_ant_pre(self._h, _ptr(t), _ptr(lens), _ptr(chk), _ptr(nchk))
        if rc != 0:
            raise ValueError("keep_pre_ls was not set")
        return t, lens, [chk[i, :nchk[i]].copy() for i in range(m)]

    def set_threads(self, threads: int) -> None:
        if self._L.orc_set_threads(self._h, int(threads)) != 0:
            raise ValueError("threads must be >= 1")

    def set_state(self, tau=None, src_route=None):
        tau = None if tau is None else np.ascontiguousarray(tau, dtype=np.float32)
        src = None if src_route is None else np.ascontiguousarray(src_route, dtype=np.int32)
        self._L.orc_set_state(self._h, _ptr(tau), _ptr(src))
