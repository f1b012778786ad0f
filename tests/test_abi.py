"""The C-ABI library without a GPU: it loads, exports every function that
include/faco.h declares, and rejects invalid arguments before touching the
device.  Without a GPU a valid call fails loudly (FACO_E_CUDA), never falls
back to the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2203_02228_gb300 import _lib, build, faco_params, params_default

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:int|void|const char\*)\s+(faco_\w+)\s*\(", src, flags=re.M))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "faco_create" in names and "faco_iterate" in names and "faco_best" in names
    assert "faco_batch_create" in names and "faco_batch_iterate" in names and "faco_batch_best" in names
    for name in names:
        assert hasattr(lib, name), name


def test_params_struct_matches_defaults(lib):
    p = params_default()
    assert p.seed == 1 and p.rho == np.float32(0.5) and p.min_new_edges == 8 and p.bl_size == 64
    assert p.p_best == 0.05 and p.p_source_gb == 0.01 and p.oropt == 1 and p.verify_pass == 1
    assert p.seg_cap == -1 and p.local_search == 1 and p.init_3opt == 0
    assert ctypes.sizeof(faco_params) == 80  # the C layout of include/faco.h on LP64


def test_invalid_arguments_are_rejected(lib):
    xy = np.zeros((10, 2), np.int32)
    xy[:, 0] = np.arange(10)
    h = ctypes.c_void_p()
    P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    assert lib.faco_create(P(xy), 2, 16, ctypes.byref(h)) == _lib.FACO_E_ARG  # n < 3
    assert lib.faco_create(P(xy), 10, 1, ctypes.byref(h)) == _lib.FACO_E_ARG  # k < 2
    assert lib.faco_create(P(xy), 10, 33, ctypes.byref(h)) == _lib.FACO_E_ARG  # k > 32
    assert lib.faco_create(None, 10, 16, ctypes.byref(h)) == _lib.FACO_E_ARG
    bad = xy.copy()
    bad[3, 1] = 1 << 24
    assert lib.faco_create(P(bad), 10, 16, ctypes.byref(h)) == _lib.FACO_E_ARG
    bad[3, 1] = -1
    assert lib.faco_create(P(bad), 10, 16, ctypes.byref(h)) == _lib.FACO_E_ARG
    for field, val in (("rho", 1.0), ("rho", 0.0), ("p_best", 1.0), ("min_new_edges", 0),
                       ("bl_size", -1), ("bl_size", 129), ("p_source_gb", 1.5), ("local_search", 2)):
        p = params_default(**{field: val})
        assert lib.faco_create_ex(P(xy), 10, 16, ctypes.byref(p), ctypes.byref(h)) == _lib.FACO_E_ARG
    assert lib.faco_iterate(None, 4, 1) == _lib.FACO_E_ARG
    assert lib.faco_best(None, None, 0, None) == _lib.FACO_E_ARG
    assert lib.faco_strerror(_lib.FACO_E_CAPACITY).decode() == "device capacity exceeded"


def test_no_cpu_fallback_without_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    xy = np.stack([np.arange(50), np.arange(50) * 3 % 17], 1).astype(np.int32)
    h = ctypes.c_void_p()
    rc = lib.faco_create(xy.ctypes.data_as(ctypes.c_void_p), 50, 16, ctypes.byref(h))
    assert rc == _lib.FACO_E_CUDA


def _batch_args(arrays):
    ptrs = (ctypes.c_void_p * len(arrays))(*[a.ctypes.data for a in arrays])
    ns = np.array([a.shape[0] for a in arrays], np.int32)
    return ctypes.cast(ptrs, ctypes.c_void_p), ns


def test_batch_invalid_arguments_are_rejected(lib):
    a = np.stack([np.arange(20), np.arange(20) * 7 % 13], 1).astype(np.int32)
    b = np.stack([np.arange(30), np.arange(30) * 5 % 11], 1).astype(np.int32)
    h = ctypes.c_void_p()
    P = lambda x: x.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    ptrs, ns = _batch_args([a, b])
    assert lib.faco_batch_create(None, P(ns), 2, 16, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    assert lib.faco_batch_create(ptrs, None, 2, 16, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    assert lib.faco_batch_create(ptrs, P(ns), 0, 16, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    assert lib.faco_batch_create(ptrs, P(ns), 2, 1, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    assert lib.faco_batch_create(ptrs, P(ns), 2, 33, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    small = ns.copy()
    small[1] = 2
    assert lib.faco_batch_create(ptrs, P(small), 2, 16, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    big = ns.copy()
    big[0] = 262145
    assert lib.faco_batch_create(ptrs, P(big), 2, 16, None, None, ctypes.byref(h)) == _lib.FACO_E_SIZE
    # k > 16 with an instance whose list is clamped to 16 or fewer: two roulette widths
    tiny = np.stack([np.arange(12), np.arange(12)], 1).astype(np.int32)
    ptrs2, ns2 = _batch_args([a, tiny])
    assert lib.faco_batch_create(ptrs2, P(ns2), 2, 24, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    bad = b.copy()
    bad[4, 0] = 1 << 24
    ptrs3, ns3 = _batch_args([a, bad])
    assert lib.faco_batch_create(ptrs3, P(ns3), 2, 16, None, None, ctypes.byref(h)) == _lib.FACO_E_ARG
    for field, val in (("keep_ant_tours", 1), ("keep_pre_ls", 1), ("seg_cap", 64), ("rho", 1.0)):
        p = params_default(**{field: val})
        assert lib.faco_batch_create(ptrs, P(ns), 2, 16, ctypes.byref(p), None, ctypes.byref(h)) == _lib.FACO_E_ARG
    assert lib.faco_batch_iterate(None, 4, 1) == _lib.FACO_E_ARG
    assert lib.faco_batch_best(None, 0, None, 0, None) == _lib.FACO_E_ARG
    assert lib.faco_batch_set_plan(None, 0) == _lib.FACO_E_ARG


def test_batch_no_cpu_fallback_without_gpu(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    a = np.stack([np.arange(40), np.arange(40) * 7 % 13], 1).astype(np.int32)
    ptrs, ns = _batch_args([a, a])
    h = ctypes.c_void_p()
    rc = lib.faco_batch_create(ptrs, ns.ctypes.data_as(ctypes.c_void_p), 2, 16, None, None, ctypes.byref(h))
    assert rc == _lib.FACO_E_CUDA


def test_server_without_gpu_and_request_sizes(lib):
    import torch

    b1 = lib.faco_server_request_bytes(1000, 16, 8, None)
    b2 = lib.faco_server_request_bytes(2000, 16, 8, None)
    b3 = lib.faco_server_request_bytes(1000, 16, 64, None)
    assert 0 < b1 < b2 and b1 < b3
    # per-ant buffers: at least route, pos, checklist, queue, log (int32) and flags per node and ant
    assert b3 - b1 >= (64 - 8) * 1000 * 21
    assert lib.faco_server_request_bytes(1000, 16, 0, None) == -1
    assert lib.faco_server_create(1 << 20, None, None) == _lib.FACO_E_ARG
    if not torch.cuda.is_available():
        h = ctypes.c_void_p()
        assert lib.faco_server_create(1 << 20, None, ctypes.byref(h)) == _lib.FACO_E_CUDA


def test_diagnostic_calls_reject_bad_arguments(lib):
    """The L2 probe and the tuner report check their arguments before any
    device work."""
    g = ctypes.c_double()
    assert lib.faco_l2_probe(1 << 10, 10, ctypes.byref(g)) == _lib.FACO_E_ARG  # below 1 MiB
    assert lib.faco_l2_probe(48 << 20, 0, ctypes.byref(g)) == _lib.FACO_E_ARG  # no repetitions
    assert lib.faco_l2_probe(48 << 20, 10, None) == _lib.FACO_E_ARG
    cnt = ctypes.c_int32()
    assert lib.faco_batch_tuner_report(None, 4, ctypes.byref(cnt)) == _lib.FACO_E_ARG
    assert lib.faco_batch_tuner_report(None, 0, None) == _lib.FACO_E_ARG
    assert lib.faco_batch_tuner_report(None, 0, ctypes.byref(cnt)) == _lib.FACO_OK
    assert cnt.value == 0  # nothing tuned in this process (no GPU here)


def test_init_3opt_is_validated(lib):
    xy = np.zeros((10, 2), np.int32)
    xy[:, 0] = np.arange(10)
    p = params_default()
    p.init_3opt = 2
    h = ctypes.c_void_p()
    assert lib.faco_create_ex(xy.ctypes.data_as(ctypes.c_void_p), 10, 4, ctypes.byref(p),
                              ctypes.byref(h)) == _lib.FACO_E_ARG
