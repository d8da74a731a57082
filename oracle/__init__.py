"""Serial CPU oracle for blocked Floyd-Warshall APSP (arXiv 1811.01201).

TEST INFRASTRUCTURE ONLY. This package is the slow, obviously correct
restatement of the method that the CUDA library is checked against. Only the
test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline /
reference arm may import it; the library (``paper_1811_01201_gb300``) never
does, and the two share no code.

The arithmetic lives in ``apsp_oracle.c`` (plain C, fp32 round-to-nearest,
built with ``-ffp-contract=off``); this module only builds it with gcc and
marshals numpy arrays through ctypes.

Functions and the passages they follow:

* ``fw_naive``    -- Section 3, Fig. 1: N rounds of k, relax all (i, j).
* ``fw_blocked``  -- Section 4.1, Fig. 2-3: R = ceil(N/BS) rounds, each in the
  four phases (diagonal block, row blocks, column blocks, the rest), every
  block updated by FW_BLOCK with a strict '<' (Section 4.2).
* ``dijkstra`` / ``bellman_ford`` -- textbook single-source shortest paths in
  double precision; pins for the two above, not part of the paper's method.
* ``path`` / ``check_paths`` -- walk of P (Section 3: P[i][j] is the most
  recently added intermediate vertex) and its validity check.
* ``check_invariants`` / ``check_bellman_row`` -- properties every exact APSP
  result has (zero diagonal, D <= W, triangle inequality, optimality).

Parity status: every function above is pinned by ``tests/test_oracle.py``
(brute force on tiny graphs, scipy's independent Floyd-Warshall and Dijkstra,
closed forms on path and complete graphs, the BS=1 / BS>=n special cases, and
planted-mistake checks). Nothing here is "parity unpinned".
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "apsp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fexcess-precision=standard", "-fPIC",
           "-shared", "-Wall"]
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile apsp_oracle.c into liboracle.so next to it (gcc, no CUDA)."""
    with _lock:
        stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "apsp_oracle.h")))
        if force or stale:
            tmp = _LIB_PATH + f".tmp{os.getpid()}"
            subprocess.run(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm"], check=True, cwd=_HERE)
            os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        f32p = ctypes.POINTER(ctypes.c_float)
        i32p = ctypes.POINTER(ctypes.c_int32)
        f64p = ctypes.POINTER(ctypes.c_double)
        c_int, c_i64, c_dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_double
        lib.oracle_fw_naive.argtypes = [f32p, c_int, f32p, i32p]
        lib.oracle_fw_naive.restype = None
        lib.oracle_fw_blocked.argtypes = [f32p, c_int, c_int, f32p, i32p]
        lib.oracle_fw_blocked.restype = None
        lib.oracle_dijkstra.argtypes = [f32p, c_int, c_int, f64p]
        lib.oracle_dijkstra.restype = None
        lib.oracle_bellman_ford.argtypes = [f32p, c_int, c_int, f64p]
        lib.oracle_bellman_ford.restype = None
        lib.oracle_path.argtypes = [i32p, c_int, c_int, c_int, i32p, c_int]
        lib.oracle_path.restype = c_int
        lib.oracle_check_paths.argtypes = [f32p, f32p, i32p, c_int, i32p, c_i64, c_dbl]
        lib.oracle_check_paths.restype = c_i64
        lib.oracle_check_invariants.argtypes = [f32p, f32p, c_int, c_dbl]
        lib.oracle_check_invariants.restype = c_i64
        lib.oracle_check_bellman_row.argtypes = [f32p, f32p, c_int, c_dbl]
        lib.oracle_check_bellman_row.restype = c_i64
        _lib = lib
    return _lib


def _f32(a: np.ndarray) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _square(W: np.ndarray) -> int:
    if W.ndim != 2 or W.shape[0] != W.shape[1]:
        raise ValueError("W must be a square matrix")
    return int(W.shape[0])


def fw_naive(W: np.ndarray):
    """Naive Floyd-Warshall (Section 3, Fig. 1). Returns (D fp32, P int32)."""
    W = _f32(W)
    n = _square(W)
    D = np.empty_like(W)
    P = np.empty((n, n), dtype=np.int32)
    _load().oracle_fw_naive(_ptr(W, ctypes.c_float), n, _ptr(D, ctypes.c_float), _ptr(P, ctypes.c_int32))
    return D, P


def fw_blocked(W: np.ndarray, bs: int):
    """Blocked Floyd-Warshall with block size ``bs`` (Section 4.1, Fig. 2-3).

    Returns (D fp32, P int32); P holds global vertex indices, -1 = none."""
    W = _f32(W)
    n = _square(W)
    if bs < 1:
        raise ValueError("bs must be >= 1")
    D = np.empty_like(W)
    P = np.empty((n, n), dtype=np.int32)
    _load().oracle_fw_blocked(_ptr(W, ctypes.c_float), n, int(bs), _ptr(D, ctypes.c_float),
                              _ptr(P, ctypes.c_int32))
    return D, P


def dijkstra(W: np.ndarray, src: int) -> np.ndarray:
    """Exact (double precision) single-source distances by dense Dijkstra."""
    W = _f32(W)
    n = _square(W)
    out = np.empty(n, dtype=np.float64)
    _load().oracle_dijkstra(_ptr(W, ctypes.c_float), n, int(src), _ptr(out, ctypes.c_double))
    return out


def bellman_ford(W: np.ndarray, src: int) -> np.ndarray:
    """Exact (double precision) single-source distances by Bellman-Ford."""
    W = _f32(W)
    n = _square(W)
    out = np.empty(n, dtype=np.float64)
    _load().oracle_bellman_ford(_ptr(W, ctypes.c_float), n, int(src), _ptr(out, ctypes.c_double))
    return out


def path(P: np.ndarray, i: int, j: int, cap: int | None = None):
    """Vertices of the path i -> j encoded in P (at most cap, default n), or None if the walk
    is malformed or longer."""
    P = np.ascontiguousarray(P, dtype=np.int32)
    n = _square(P)
    cap = n if cap is None else int(cap)
    out = np.empty(max(cap, 1), dtype=np.int32)
    cnt = _load().oracle_path(_ptr(P, ctypes.c_int32), n, int(i), int(j), _ptr(out, ctypes.c_int32), cap)
    return None if cnt < 0 else [int(v) for v in out[:cnt]]


def check_paths(W: np.ndarray, D: np.ndarray, P: np.ndarray, pairs: np.ndarray, rtol: float = 0.0) -> int:
    """Number of (i, j) pairs whose P-walk is not a simple path of weight D[i][j]."""
    W = _f32(W)
    D = _f32(D)
    P = np.ascontiguousarray(P, dtype=np.int32)
    n = _square(W)
    pairs = np.ascontiguousarray(pairs, dtype=np.int32).reshape(-1, 2)
    return int(_load().oracle_check_paths(_ptr(W, ctypes.c_float), _ptr(D, ctypes.c_float),
                                          _ptr(P, ctypes.c_int32), n, _ptr(pairs, ctypes.c_int32),
                                          int(pairs.shape[0]), float(rtol)))


def check_invariants(W: np.ndarray, D: np.ndarray, rtol: float = 0.0) -> int:
    """Violations of D[i][i]==0, D<=W and the triangle inequality (O(n^3))."""
    W = _f32(W)
    D = _f32(D)
    n = _square(W)
    return int(_load().oracle_check_invariants(_ptr(W, ctypes.c_float), _ptr(D, ctypes.c_float), n,
                                               float(rtol)))


def check_bellman_row(W: np.ndarray, Drow: np.ndarray, rtol: float = 0.0) -> int:
    """Violations of the optimality condition D[s][j] <= D[s][k] + W[k][j]."""
    W = _f32(W)
    n = _square(W)
    Drow = np.ascontiguousarray(Drow, dtype=np.float32).reshape(n)
    return int(_load().oracle_check_bellman_row(_ptr(W, ctypes.c_float), _ptr(Drow, ctypes.c_float), n,
                                                float(rtol)))
