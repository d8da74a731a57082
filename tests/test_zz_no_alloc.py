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


class _Mempool:
    """Usage counters of the device's default stream-ordered memory pool, read through the CUDA
    driver API (the pool is a driver object, whichever runtime copy asks)."""

    RESERVED_MEM_CURRENT, USED_MEM_CURRENT, USED_MEM_HIGH = 5, 7, 8  # CUmemPool_attribute

    def __init__(self):
        self.cu = ctypes.CDLL("libcuda.so.1")
        dev = ctypes.c_int()
        assert self.cu.cuDeviceGet(ctypes.byref(dev), torch.cuda.current_device()) == 0
        self.pool = ctypes.c_void_p()
        assert self.cu.cuDeviceGetDefaultMemPool(ctypes.byref(self.pool), dev) == 0

    def get(self, attr: int) -> int:
        v = ctypes.c_uint64()
        assert self.cu.cuMemPoolGetAttribute(self.pool, attr, ctypes.byref(v)) == 0
        return int(v.value)

    def reset_high(self):
        zero = ctypes.c_uint64(0)
        assert self.cu.cuMemPoolSetAttribute(self.pool, self.USED_MEM_HIGH, ctypes.byref(zero)) == 0


def test_noalloc_allocates_no_device_memory():
    # The property the entry point exists for: a call takes nothing from the stream-ordered pool
    # (not even briefly: the pool's high-water mark does not move) and nothing from the device's
    # free memory. The first call on a device may load the library's module (with its fixed
    # array); the checks start after it.
    L = _lib()
    n = 1024
    Wd = inputs.dense_digraph(n, 14, 1, 1000, density=0.5, device=DEV)
    D = torch.empty_like(Wd)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    o = apsp.apsp_options(64, apsp.DTYPE_AUTO, 1, 0)
    s = torch.cuda.current_stream()

    def call():
        st = L.apsp_fw_noalloc(Wd.data_ptr(), D.data_ptr(), P.data_ptr(), n, ctypes.byref(o), None, s.cuda_stream)
        torch.cuda.synchronize()
        assert st == apsp.APSP_OK, apsp.status_str(st)

    call()
    pool = _Mempool()
    for _ in range(2):
        used, reserved = pool.get(pool.USED_MEM_CURRENT), pool.get(pool.RESERVED_MEM_CURRENT)
        pool.reset_high()
        free_before = torch.cuda.mem_get_info()[0]
        call()
        free_after = torch.cuda.mem_get_info()[0]
        assert pool.get(pool.USED_MEM_HIGH) <= used, "the call took memory from the stream-ordered pool"
        assert pool.get(pool.USED_MEM_CURRENT) == used and pool.get(pool.RESERVED_MEM_CURRENT) == reserved
        assert free_after == free_before, "the device's free memory changed across the call"
    # the same measurement sees the allocating entry point take its workspace from the pool
    pool.reset_high()
    used = pool.get(pool.USED_MEM_CURRENT)
    apsp.apsp_fw_ex(Wd, D, P, bs=64)
    torch.cuda.synchronize()
    assert pool.get(pool.USED_MEM_HIGH) > used


def test_noalloc_sizes_misaligned_matrices_before_enqueueing():
    # a D that does not start on a 16-byte boundary needs a padded working copy in the fixed
    # array; the entry point sizes for the D and P it is given. n = 2048: the copy fits and the
    # result equals the allocating entry point's; n = 4096: it fits only when aligned, and the
    # call is refused with APSP_ENOMEM before anything is enqueued (D keeps its contents).
    L = _lib()
    cap = L.apsp_noalloc_scratch_bytes()
    o = apsp.apsp_options(64, apsp.DTYPE_F32, 1, 0)
    for n in (2048, 4096):
        assert apsp.apsp_fw_workspace_size(n, bs=64, dtype=apsp.DTYPE_F32) <= cap
        Wd = inputs.dense_digraph(n, 15, 1, 1000, device=DEV)
        buf = torch.full((n * n + 1,), -3.0, device=DEV)
        Dm = buf[1:]  # 4-byte offset
        P = torch.empty((n, n), dtype=torch.int32, device=DEV)
        need = apsp.apsp_fw_workspace_size_for(n, Dm.data_ptr(), P.data_ptr(), bs=64, dtype=apsp.DTYPE_F32)
        assert need == apsp.apsp_fw_workspace_size(n, bs=64, dtype=apsp.DTYPE_F32) + 4 * n * n
        st = L.apsp_fw_noalloc(Wd.data_ptr(), Dm.data_ptr(), P.data_ptr(), n, ctypes.byref(o), None,
                               torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        if need > cap:
            assert n == 4096 and st == apsp.APSP_ENOMEM
            assert bool((Dm == -3.0).all())
        else:
            assert n == 2048 and st == apsp.APSP_OK, apsp.status_str(st)
            Dr, Pr = _reference(Wd, 64, apsp.DTYPE_F32)
            assert torch.equal(Dm.view(n, n), Dr) and torch.equal(P, Pr)
