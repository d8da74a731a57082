"""CPU-side checks of the C ABI: the library builds, loads, and exports every
function that include/apsp.h declares. No compute calls (no GPU here)."""

import ctypes
import os
import re

import numpy as np
import pytest

import paper_1811_01201_gb300 as apsp
from paper_1811_01201_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if not f.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", f)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(apsp_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


def test_library_builds_and_loads():
    path = _build.build()
    assert os.path.exists(path)
    lib = ctypes.CDLL(path)
    assert lib is not None


def test_every_declared_symbol_is_exported():
    lib = ctypes.CDLL(_build.build())
    declared = _declared_functions()
    assert {"apsp_fw", "apsp_fw_ex", "apsp_fw_batched", "apsp_serve_create", "apsp_path"} <= declared
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, f"declared in include/*.h but not exported: {missing}"


def test_host_only_helpers():
    # these touch no GPU state
    assert apsp.apsp_default_bs(512) in (32, 64, 128)
    assert apsp.status_str(apsp.APSP_EINVAL) == "invalid argument"
    assert apsp.apsp_fw_workspace_size(128, dtype=apsp.DTYPE_F32) >= 256
    assert apsp.apsp_fw_workspace_size(100, dtype=apsp.DTYPE_F32) >= 128 * 128 * 8
    assert apsp.apsp_fw_workspace_size(0) == 0


def test_workspace_size_formula():
    # documented in include/apsp.h: a 256-byte head, the round's packed panel slices
    # (fp32: ceil(n/128) * bs * 1072 bytes; 16-bit: * 800) and the packed diagonal block
    # (8 * bs * (bs + 4) bytes), each rounded up to 256 bytes; n*n working matrices only
    # when n is not a multiple of 128 (fp32) or for the 16-bit path
    def up(x):
        return (x + 255) // 256 * 256
    for n, bs in [(128, 32), (1024, 64), (32768, 64), (65536, 64), (4096, 128)]:
        nt = n // 128
        want = 256 + up(nt * bs * 1072) + up(8 * bs * (bs + 4))
        assert apsp.apsp_fw_workspace_size(n, bs=bs, dtype=apsp.DTYPE_F32) == want, (n, bs)
    n, bs = 4096, 64  # 16-bit: D16 working matrix, P in place
    want16 = 256 + up(2 * n * n) + up((n // 128) * bs * 800) + up(8 * bs * (bs + 4))
    f32 = 256 + up((n // 128) * bs * 1072) + up(8 * bs * (bs + 4))
    assert apsp.apsp_fw_workspace_size(n, bs=bs) == max(want16, f32)
    # default block size: 64 on the fp32 path above n = 512, 128 on the 16-bit path above 16384
    assert apsp.apsp_fw_workspace_size(40000 // 128 * 128, dtype=apsp.DTYPE_F32) == \
        apsp.apsp_fw_workspace_size(40000 // 128 * 128, bs=64, dtype=apsp.DTYPE_F32)
    big = 20480
    assert apsp.apsp_fw_workspace_size(big) == max(
        apsp.apsp_fw_workspace_size(big, bs=64, dtype=apsp.DTYPE_F32),
        256 + up(2 * big * big) + up((big // 128) * 128 * 800) + up(8 * 128 * 132))


def test_workspace_size_for_misaligned_matrices():
    # the solve runs in place only in 16-byte-aligned D and P; a misaligned one needs its padded
    # working copy (4 * n_pad^2 bytes) in the workspace, and apsp_fw_ex checks this before it
    # enqueues anything
    n, bs = 1024, 64
    base = apsp.apsp_fw_workspace_size(n, bs=bs, dtype=apsp.DTYPE_F32)
    assert apsp.apsp_fw_workspace_size_for(n, 0x10000, 0x20000, bs=bs, dtype=apsp.DTYPE_F32) == base
    extra = 4 * n * n
    assert apsp.apsp_fw_workspace_size_for(n, 0x10004, 0x20000, bs=bs, dtype=apsp.DTYPE_F32) == base + extra
    assert apsp.apsp_fw_workspace_size_for(n, 0x10000, 0x20008, bs=bs, dtype=apsp.DTYPE_F32) == base + extra
    assert apsp.apsp_fw_workspace_size_for(n, 0x10004, 0x20008, bs=bs, dtype=apsp.DTYPE_F32) == base + 2 * extra
    # n not a multiple of 128: working copies either way, alignment changes nothing
    m = 1000
    assert apsp.apsp_fw_workspace_size_for(m, 0x10004, 0x20008, bs=bs, dtype=apsp.DTYPE_F32) == \
        apsp.apsp_fw_workspace_size(m, bs=bs, dtype=apsp.DTYPE_F32)
    # AUTO takes the larger of the two arithmetics for the same pointers
    assert apsp.apsp_fw_workspace_size_for(n, 0x10004, 0x20000, bs=bs) >= base + extra


def test_path_helper_matches_oracle_walk():
    import oracle
    from paper_1811_01201_gb300 import inputs
    n = 70
    W = inputs.dense_digraph(n, 3, 1, 50, density=0.3).numpy()
    D, P = oracle.fw_blocked(W, 16)
    for i in range(0, n, 7):
        for j in range(0, n, 5):
            assert apsp.apsp_path(P, i, j) == oracle.path(P, i, j)
    bad = P.copy()
    bad[0, 1] = 0  # intermediate equal to an endpoint
    assert apsp.apsp_path(bad, 0, 1) is None
    # a capacity below the path's vertex count fails; exactly the count succeeds
    for i, j in [(0, 69), (5, 33), (60, 2)]:
        full = oracle.path(P, i, j)
        assert apsp.apsp_path(P, i, j, cap=len(full)) == full
        assert apsp.apsp_path(P, i, j, cap=len(full) - 1) is None
        assert oracle.path(P, i, j, cap=len(full) - 1) is None


def test_path_helper_matches_oracle_on_malformed_matrices():
    import oracle
    # random P over [-1, n): cycles, self-references and long walks; host helper and oracle
    # agree on every pair and capacity (both the vertex list and the failure)
    rng = np.random.default_rng(4)
    for trial in range(30):
        n = int(rng.integers(2, 12))
        P = rng.integers(-1, n, size=(n, n)).astype(np.int32)
        if trial % 3 == 0:
            P[rng.random((n, n)) < 0.6] = -1
        for cap in (1, 2, 3, 5, n, 2 * n):
            for i in range(n):
                for j in range(n):
                    assert apsp.apsp_path(P, i, j, cap) == oracle.path(P, i, j, cap), (trial, cap, i, j)


def test_argument_checks_return_status_without_touching_the_gpu():
    # every one of these is rejected by host-side validation before any CUDA call
    L = apsp.load()
    vp = ctypes.c_void_p
    assert L.apsp_fw(None, None, None, 16, None) == apsp.APSP_EINVAL
    o = apsp.apsp_options(48, 0, 1, 0)
    assert L.apsp_fw_ex(None, None, None, 0, ctypes.byref(o), None, 0, None, None) == apsp.APSP_EINVAL
    assert L.apsp_batch_create(None, None, None, None, 0, None, ctypes.byref(vp()), None) == apsp.APSP_EINVAL
    assert L.apsp_batch_launch(None, None) == apsp.APSP_EINVAL
    assert L.apsp_batch_autotune(None, None, None) == apsp.APSP_EINVAL
    assert L.apsp_serve_create(None, 1 << 30, 4) == apsp.APSP_EINVAL
    h = vp()
    assert L.apsp_serve_create(ctypes.byref(h), 1 << 30, 0) == apsp.APSP_EINVAL
    assert L.apsp_serve_submit(None, None, 10, None) == apsp.APSP_EINVAL
    assert L.apsp_serve_poll(None, 1, None, None, None, 0) == apsp.APSP_EINVAL
    assert L.apsp_serve_stats(None, None) == apsp.APSP_EINVAL
    assert L.apsp_serve_destroy(None) == apsp.APSP_EINVAL
    assert L.apsp_batched_bs(100) == 32
    fake = ctypes.c_void_p(256)
    assert L.apsp_paths(fake, 0, fake, 4, fake, 8, fake, None) == apsp.APSP_EINVAL     # n < 1
    assert L.apsp_paths(fake, 16, fake, -1, fake, 8, fake, None) == apsp.APSP_EINVAL   # count < 0
    assert L.apsp_paths(fake, 16, fake, 4, fake, 0, fake, None) == apsp.APSP_EINVAL    # cap < 1
    assert L.apsp_paths(fake, 16, None, 4, fake, 8, fake, None) == apsp.APSP_EINVAL    # null pairs
    assert L.apsp_paths(None, 16, None, 0, None, 8, None, None) == apsp.APSP_OK        # nothing to do


def test_size_limits_rejected_on_the_host():
    # non-null placeholder pointers: the checks on n and options come before any CUDA call
    L = apsp.load()
    fake = ctypes.c_void_p(256)
    o = apsp.apsp_options(0, apsp.DTYPE_F32, 0, 0)
    assert L.apsp_fw_ex(fake, fake, fake, 65537, ctypes.byref(o), None, 0, None, None) == apsp.APSP_EINVAL
    assert L.apsp_fw_ex(fake, fake, fake, -5, ctypes.byref(o), None, 0, None, None) == apsp.APSP_EINVAL
    o_bad = apsp.apsp_options(0, 7, 1, 0)  # unknown dtype
    assert L.apsp_fw_ex(fake, fake, fake, 64, ctypes.byref(o_bad), None, 0, None, None) == apsp.APSP_EINVAL
    o_u16 = apsp.apsp_options(0, apsp.DTYPE_U16X2, 0, 0)  # 16-bit needs the validation scan
    assert L.apsp_fw_ex(fake, fake, fake, 64, ctypes.byref(o_u16), None, 0, None, None) == apsp.APSP_EINVAL
    # misaligned caller workspace
    assert L.apsp_fw_ex(fake, fake, fake, 64, ctypes.byref(o), ctypes.c_void_p(4096 + 8), 1 << 20, None,
                        None) == apsp.APSP_EINVAL
    n_arr = (ctypes.c_int * 1)(513)
    ptrs = (ctypes.c_void_p * 1)(256)
    out = ctypes.c_void_p()
    assert L.apsp_batch_create(ptrs, ptrs, ptrs, n_arr, 1, None, ctypes.byref(out), None) == apsp.APSP_EINVAL
