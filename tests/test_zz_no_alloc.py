"""faco_lists_noalloc: candidate lists for callers that may not allocate
device memory (a pooled or framework-owned device, or a loop that cannot
take the synchronisation cudaMalloc/cudaFree bring).  The call must give
the same lists as the allocating path (faco_create + faco_get_lists), on two
calls in a row -- the second one reusing the library's fixed scratch array
after the first left it dirty.  Kept in a file collected last."""
import ctypes

import numpy as np
import pytest

from paper_2203_02228_gb300 import Colony, _lib, inputs

pytestmark = pytest.mark.gpu


def lists_noalloc(xy, k=16, bl=64):
    import torch

    L = _lib.load()
    L.faco_lists_noalloc.restype = ctypes.c_int
    L.faco_lists_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    n = xy.shape[0]
    ke = min(k, n - 1)
    ble = min(bl, n - 1 - ke)
    dev = torch.device("cuda", 0)
    xy_d = torch.from_numpy(np.ascontiguousarray(xy, dtype=np.int32)).to(dev)
    cand = torch.empty(n * ke, dtype=torch.int32, device=dev)
    backup = torch.empty(max(n * ble, 1), dtype=torch.int32, device=dev)
    eta = torch.empty(n * ke, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = L.faco_lists_noalloc(xy_d.data_ptr(), n, k, bl, cand.data_ptr(), backup.data_ptr(), eta.data_ptr(),
                              stream.cuda_stream)
    assert rc == 0, _lib.strerror(rc)
    torch.cuda.synchronize(dev)
    return (cand.cpu().numpy().reshape(n, ke), backup.cpu().numpy()[:n * ble].reshape(n, ble),
            eta.cpu().numpy().reshape(n, ke))


def test_noalloc_lists_match_allocating_path_twice():
    first = inputs.stippled(6000, seed=61, blobs=12, ridges=3, side=80000)
    second = inputs.uniform(2500, seed=62)
    for xy in (first, second):
        got = lists_noalloc(xy)
        want = Colony(xy, 16).lists()
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_array_equal(got[1], want[1])
        assert np.array_equal(got[2].view(np.uint32), want[2].view(np.uint32))


def test_noalloc_rejects_sizes_beyond_its_scratch():
    L = _lib.load()
    L.faco_lists_noalloc.restype = ctypes.c_int
    L.faco_lists_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    dummy = ctypes.c_void_p(16)  # never dereferenced: the size check comes first
    assert L.faco_lists_noalloc(dummy, (1 << 18) + 1, 16, 64, dummy, dummy, dummy, None) == _lib.FACO_E_SIZE
