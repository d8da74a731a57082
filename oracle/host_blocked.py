"""ctypes wrapper of host_blocked.c: the paper's blocked design (Section 4) on the host cores.

CPU baseline for the benchmark, pinned bit for bit to ``oracle.fw_blocked`` by the tests;
test and benchmark infrastructure only. Built with gcc and OpenMP when the compiler has it,
else serial (``threads()`` reports which).
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "host_blocked.c")
_LIB_PATH = os.path.join(_HERE, "libhostblocked.so")
_CFLAGS = ["-O3", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-Wall"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile host_blocked.c into libhostblocked.so (gcc; OpenMP if available)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            try:
                subprocess.run(["gcc", *_CFLAGS, "-fopenmp", "-o", tmp, _SRC], check=True, cwd=_HERE,
                               capture_output=True)
            except subprocess.CalledProcessError:
                subprocess.run(["gcc", *_CFLAGS, "-Wno-unknown-pragmas", "-o", tmp, _SRC], check=True, cwd=_HERE)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.host_fw_blocked.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)]
        lib.host_fw_blocked.restype = None
        lib.host_fw_blocked_threads.argtypes = []
        lib.host_fw_blocked_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """Threads the parallel loops use (OMP_NUM_THREADS, else all host cores; 1 without OpenMP)."""
    return int(_load().host_fw_blocked_threads())


def fw_blocked(W: np.ndarray, bs: int = 64):
    """Blocked Floyd-Warshall on the host cores; returns (D fp32, P int32) equal to
    ``oracle.fw_blocked(W, bs)``."""
    W = np.ascontiguousarray(W, dtype=np.float32)
    if W.ndim != 2 or W.shape[0] != W.shape[1]:
        raise ValueError("W must be a square matrix")
    if bs < 1:
        raise ValueError("bs must be >= 1")
    n = int(W.shape[0])
    D = np.empty_like(W)
    P = np.empty((n, n), dtype=np.int32)
    f32p, i32p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
    _load().host_fw_blocked(W.ctypes.data_as(f32p), n, int(bs), D.ctypes.data_as(f32p), P.ctypes.data_as(i32p))
    return D, P
