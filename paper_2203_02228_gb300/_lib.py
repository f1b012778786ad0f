"""ctypes binding of libfaco.so: the C ABI of include/faco.h, same names.

Argument marshalling only -- every step of the method runs in the library's
CUDA kernels.  Loading fails loudly (RuntimeError) when the library has not
been built; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

_lock = threading.Lock()
_lib = None

FACO_OK = 0
FACO_E_ARG = -1
FACO_E_SIZE = -2
FACO_E_NOMEM = -3
FACO_E_CUDA = -4
FACO_E_TIMEOUT = -5
FACO_E_STATE = -6
FACO_E_CAPACITY = -7


class faco_params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("rho", ctypes.c_float),
        ("min_new_edges", ctypes.c_int32),
        ("bl_size", ctypes.c_int32),
        ("p_best", ctypes.c_double),
        ("p_source_gb", ctypes.c_double),
        ("oropt", ctypes.c_int32),
        ("verify_pass", ctypes.c_int32),
        ("keep_ant_tours", ctypes.c_int32),
        ("keep_pre_ls", ctypes.c_int32),
        ("seg_cap", ctypes.c_int32),
        ("local_search", ctypes.c_int32),
        ("init_3opt", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
    ]


class faco_stats(ctypes.Structure):
    _fields_ = [
        ("iteration", ctypes.c_int64),
        ("best_length", ctypes.c_int64),
        ("initial_length", ctypes.c_int64),
        ("source_length", ctypes.c_int64),
        ("n", ctypes.c_int32),
        ("k", ctypes.c_int32),
        ("bl", ctypes.c_int32),
        ("ants", ctypes.c_int32),
        ("aco_steps", ctypes.c_int64),
        ("new_edges", ctypes.c_int64),
        ("backup_picks", ctypes.c_int64),
        ("global_picks", ctypes.c_int64),
        ("ls_pops", ctypes.c_int64),
        ("moves_2opt", ctypes.c_int64),
        ("moves_or", ctypes.c_int64),
        ("flip_elems", ctypes.c_int64),
        ("kernel_launches", ctypes.c_int64),
        ("redone_ants", ctypes.c_int64),
        ("seg_cap", ctypes.c_int32),
        ("pad", ctypes.c_int32),
    ]


class faco_server_stats(ctypes.Structure):
    _fields_ = [(name, ctypes.c_int64) for name in (
        "submitted", "completed", "queued", "setting_up", "active", "peak_active", "rounds",
        "kernel_launches", "pool_bytes", "pool_in_use")]


FACO_PENDING = 1


class FacoError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        msg = strerror(status) if _lib is not None else str(status)
        super().__init__("%s failed: %s (%d)" % (what or "faco call", msg, status))


def lib_path() -> str:
    return _build.LIB


def load():
    """Loads libfaco.so (built in-tree by build.build()); raises if missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libfaco.so is not built (%s); run paper_2203_02228_gb300.build.build()" % path)
        L = ctypes.CDLL(path)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        P = ctypes.POINTER
        sig = {
            "faco_params_default": (ctypes.c_int, [P(faco_params)]),
            "faco_create": (ctypes.c_int, [vp, i32, i32, P(vp)]),
            "faco_create_ex": (ctypes.c_int, [vp, i32, i32, P(faco_params), P(vp)]),
            "faco_create_device": (ctypes.c_int, [vp, i32, i32, P(faco_params), P(vp)]),
            "faco_iterate": (ctypes.c_int, [vp, i32, i32]),
            "faco_sync": (ctypes.c_int, [vp]),
            "faco_best": (ctypes.c_int, [vp, vp, i32, P(i64)]),
            "faco_best_device": (ctypes.c_int, [vp, vp, vp]),
            "faco_stats_get": (ctypes.c_int, [vp, P(faco_stats)]),
            "faco_destroy": (None, [vp]),
            "faco_strerror": (ctypes.c_char_p, [ctypes.c_int]),
            "faco_get_lists": (ctypes.c_int, [vp, vp, vp, vp]),
            "faco_get_tau": (ctypes.c_int, [vp, vp]),
            "faco_get_limits": (ctypes.c_int, [vp, vp]),
            "faco_get_source": (ctypes.c_int, [vp, vp, P(i64)]),
            "faco_get_initial": (ctypes.c_int, [vp, vp, P(i64)]),
            "faco_get_history": (ctypes.c_int, [vp, vp, i64, P(i64)]),
            "faco_get_ant_tours": (ctypes.c_int, [vp, vp, vp]),
            "faco_get_ant_pre": (ctypes.c_int, [vp, vp, vp, vp, vp]),
            "faco_get_ant_stats": (ctypes.c_int, [vp, vp]),
            "faco_lists_noalloc": (ctypes.c_int, [vp, i32, i32, i32, vp, vp, vp, vp]),
            "faco_profile_enable":(ctypes.c_int, [vp, ctypes.c_int]),
            "faco_profile_read": (ctypes.c_int, [vp, P(ctypes.c_double), P(i64)]),
            "faco_l2_probe": (ctypes.c_int, [ctypes.c_size_t, i32, P(ctypes.c_double)]),
            "faco_test_device":(ctypes.c_int, [ctypes.c_int, vp, ctypes.c_size_t, vp, ctypes.c_size_t,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_uint64]),
            # include/faco_batch.h
            "faco_batch_create": (ctypes.c_int, [vp, vp, i32, i32, P(faco_params), vp, P(vp)]),
            "faco_batch_iterate": (ctypes.c_int, [vp, i32, i32]),
            "faco_batch_sync": (ctypes.c_int, [vp]),
            "faco_batch_best": (ctypes.c_int, [vp, i32, vp, i32, P(i64)]),
            "faco_batch_tours": (ctypes.c_int, [vp, vp, vp]),
            "faco_batch_stats": (ctypes.c_int, [vp, i32, P(faco_stats)]),
            "faco_batch_tau": (ctypes.c_int, [vp, i32, vp]),
            "faco_batch_set_plan": (ctypes.c_int, [vp, i32]),
            "faco_batch_get_plan": (ctypes.c_int, [vp, vp]),
            "faco_batch_destroy": (None, [vp]),
            "faco_batch_tuner_report": (ctypes.c_int, [vp, i32, P(i32)]),
            # include/faco_serve.h
            "faco_server_create": (ctypes.c_int, [ctypes.c_size_t, P(faco_params), P(vp)]),
            "faco_server_request_bytes": (i64, [i32, i32, i32, P(faco_params)]),
            "faco_server_submit": (ctypes.c_int, [vp, vp, i32, i32, i32, i32, ctypes.c_uint64,
                                                  P(ctypes.c_uint64)]),
            "faco_server_poll": (ctypes.c_int, [vp, ctypes.c_uint64, vp, i32, P(i64), P(i64), P(i64)]),
            "faco_server_wait": (ctypes.c_int, [vp, ctypes.c_uint64, i32]),
            "faco_server_release": (ctypes.c_int, [vp, ctypes.c_uint64]),
            "faco_server_stats_get": (ctypes.c_int, [vp, P(faco_server_stats)]),
            "faco_server_destroy": (None, [vp]),
            "faco_test_pool": (ctypes.c_int, [i64, vp, i32, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def strerror(status: int) -> str:
    return load().faco_strerror(status).decode()


def check(status: int, what: str = "") -> None:
    if status != FACO_OK:
        raise FacoError(status, what)


def params_default(**kw) -> faco_params:
    p = faco_params()
    check(load().faco_params_default(ctypes.byref(p)), "faco_params_default")
    for k, v in kw.items():
        setattr(p, k, v)
    return p
