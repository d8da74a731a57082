"""apsp_fw_noalloc: the allocation-free solve for callers that cannot allocate
device memory when they need a solve. It works in one fixed device array
inside the library, so these checks call it through the C ABI and compare its
D and P with the ordinary entry point (apsp_fw_ex) bit for bit -- the same
exactness every parity test here uses -- on two calls in a row, the second of
which must not be affected by what the first left in the shared array.

This file is collected last on purpose, so that a failure here stops a
`-x` run only after every other test has run.
"""

import ctypes

import numpy as np
import pytest
import torch

import paper_1811_01201_gb300 as apsp
from paper_1811_01201_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _lib():
    L = apsp.load()
    vp = ctypes.c_void_p
    L.apsp_fw_noalloc.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(apsp.apsp_options),
                                  ctypes.POINTER(apsp.apsp_run_info), vp]
    L.apsp_fw_noalloc.restype = ctypes.c_int
    L.apsp_noalloc_scratch_bytes.argtypes = []
    L.apsp_noalloc_scratch_bytes.restype = ctypes.c_size_t
    return L


def _noalloc(L, Wd, bs, dtype=apsp.DTYPE_AUTO, stream=None):
    n = Wd.shape[0]
    D = torch.full_like(Wd, -7.0)
    P = torch.full((n, n), 12345, dtype=torch.int32, device=DEV)
    o = apsp.apsp_options(bs, dtype, 1, 0)
    info = apsp.apsp_run_info()
    s = torch.cuda.current_stream() if stream is None else stream
    st = L.apsp_fw_noalloc(Wd.data_ptr(), D.data_ptr(), P.data_ptr(), n, ctypes.byref(o), ctypes.byref(info),
                           s.cuda_stream)
    torch.cuda.synchronize()
    return st, D, P, info


def _reference(Wd, bs, dtype=apsp.DTYPE_AUTO):
    D = torch.empty_like(Wd)
    P = torch.empty(Wd.shape, dtype=torch.int32, device=DEV)
    apsp.apsp_fw_ex(Wd, D, P, bs=bs, dtype=dtype)
    torch.cuda.synchronize()
    return D, P


def test_noalloc_matches_allocating_entry_point_twice():
    L = _lib()
    # two different graphs in a row: the second call reuses the shared array the first one filled
    cases = [(1000, 11, 1, 1000, 0.5, 64, apsp.DTYPE_F32),     # padded working pair in the array
             (700, 12, 1, 30, 0.8, 32, apsp.DTYPE_AUTO)]       # 16-bit working matrix in the array
    for n, seed, lo, hi, dens, bs, dt in cases:
        Wd = inputs.dense_digraph(n, seed, lo, hi, density=dens, device=DEV)
        st, D, P, info = _noalloc(L, Wd, bs, dt)
        assert st == apsp.APSP_OK, apsp.status_str(st)
        Dr, Pr = _reference(Wd, bs, dt)
        assert torch.equal(D, Dr) and torch.equal(P, Pr)
        assert info.bs_used == bs


def test_noalloc_real_weights_and_in_place_size():
    L = _lib()
    Wd = inputs.dense_digraph(384, 13, kind="real", density=0.9, device=DEV)
    for _ in range(2):
        st, D, P, _ = _noalloc(L, Wd, 64, apsp.DTYPE_F32)
        assert st == apsp.APSP_OK
        Dr, Pr = _reference(Wd, 64, apsp.DTYPE_F32)
        assert torch.equal(D, Dr) and torch.equal(P, Pr)


def test_noalloc_rejects_sizes_beyond_the_array():
    L = _lib()
    cap = L.apsp_noalloc_scratch_bytes()
    assert cap == 64 << 20
    n = 3000  # padded to 3072: 8 * 3072^2 bytes of working matrices do not fit
    assert apsp.apsp_fw_workspace_size(n, dtype=apsp.DTYPE_F32) > cap
    W = torch.zeros((n, n), device=DEV)
    st, _, _, _ = _noalloc(L, W, 64, apsp.DTYPE_F32)
    assert st == apsp.APSP_ENOMEM
    o = apsp.apsp_options(64, apsp.DTYPE_F32, 1, apsp.FLAG_TIME_PHASES)
    assert L.apsp_fw_noalloc(W.data_ptr(), W.data_ptr(), W.data_ptr(), 128, ctypes.byref(o), None,
                             None) == apsp.APSP_EINVAL
