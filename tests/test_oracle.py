"""Pins for the CPU oracle: it is checked here against things other than itself.

Every check is on the CPU. The pins are brute force on tiny graphs, closed
forms, the BS=1 / BS>=n special cases (blocked FW reduces to Fig. 1),
hand-derived fixtures under tests/golden/, scipy's independent Floyd-Warshall
and Dijkstra, and structural properties of P. The mutant tests at the end
plant plausible mistakes in a copy of the oracle and show that some pin
catches each one.
"""

import ctypes
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse.csgraph as csg

import oracle
from paper_1811_01201_gb300 import inputs
from tests.helpers import all_pairs, brute_force_apsp, load_golden, random_pairs

INF = np.float32(np.inf)


def _w(n, seed, lo=1, hi=100, density=1.0, kind="int"):
    return inputs.dense_digraph(n, seed, lo, hi, density=density, kind=kind).numpy()


def _scipy_apsp(W):
    G = csg.csgraph_from_dense(W.astype(np.float64), null_value=np.inf)
    return csg.floyd_warshall(G, directed=True)


# ---------------------------------------------------------------- golden fixtures

@pytest.mark.parametrize("name", ["tie_break_4.txt", "blocked_vs_naive_4.txt"])
def test_golden_fixtures(name):
    g = load_golden(name)
    D, P = oracle.fw_naive(g["W"])
    np.testing.assert_array_equal(D, g["D_naive"])
    np.testing.assert_array_equal(P, g["P_naive"])
    D, P = oracle.fw_blocked(g["W"], g["bs"])
    np.testing.assert_array_equal(D, g["D_blocked"])
    np.testing.assert_array_equal(P, g["P_blocked"])


# ---------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [1, 2, 3, 5, 6, 7])
@pytest.mark.parametrize("density", [1.0, 0.45])
def test_brute_force_int(n, density):
    for seed in range(4):
        W = _w(n, 100 + seed, 1, 9, density)
        ref = brute_force_apsp(W)
        D, P = oracle.fw_naive(W)
        np.testing.assert_array_equal(D.astype(np.float64), ref)
        for bs in sorted({1, 2, 3, n, n + 2}):
            Db, Pb = oracle.fw_blocked(W, bs)
            np.testing.assert_array_equal(Db.astype(np.float64), ref)
            assert oracle.check_paths(W, Db, Pb, all_pairs(n)) == 0


@pytest.mark.parametrize("n", [4, 7])
def test_brute_force_real(n):
    for seed in range(4):
        W = _w(n, 200 + seed, kind="real", density=0.7)
        ref = brute_force_apsp(W)
        for D, P in (oracle.fw_naive(W), oracle.fw_blocked(W, 2), oracle.fw_blocked(W, 3)):
            fin = np.isfinite(ref)
            assert (np.isfinite(D) == fin).all()
            np.testing.assert_allclose(D[fin], ref[fin], rtol=1e-6)


# ---------------------------------------------------------------- closed forms

@pytest.mark.parametrize("bs", [None, 1, 3, 4, 16])
def test_directed_chain(bs):
    n = 13
    W = np.full((n, n), INF, dtype=np.float32)
    np.fill_diagonal(W, 0)
    for t in range(n - 1):
        W[t, t + 1] = t + 1
    D, P = oracle.fw_naive(W) if bs is None else oracle.fw_blocked(W, bs)
    for i in range(n):
        for j in range(n):
            if i <= j:
                assert D[i, j] == sum(t + 1 for t in range(i, j))
                assert oracle.path(P, i, j) == list(range(i, j + 1))
            else:
                assert D[i, j] == INF and P[i, j] == -1


@pytest.mark.parametrize("bs", [None, 2, 5])
def test_directed_cycle(bs):
    n = 11
    W = np.full((n, n), INF, dtype=np.float32)
    np.fill_diagonal(W, 0)
    for t in range(n):
        W[t, (t + 1) % n] = 3
    D, P = oracle.fw_naive(W) if bs is None else oracle.fw_blocked(W, bs)
    for i in range(n):
        for j in range(n):
            assert D[i, j] == 3 * ((j - i) % n)
    assert oracle.check_paths(W, D, P, all_pairs(n)) == 0


@pytest.mark.parametrize("bs", [None, 1, 4])
def test_complete_unit_weights(bs):
    # every direct edge is already shortest; no strict improvement ever happens
    n = 9
    W = np.ones((n, n), dtype=np.float32)
    np.fill_diagonal(W, 0)
    D, P = oracle.fw_naive(W) if bs is None else oracle.fw_blocked(W, bs)
    np.testing.assert_array_equal(D, W)
    assert (P == -1).all()


def test_diagonal_forced_to_zero():
    W = _w(6, 7)
    np.fill_diagonal(W, 5.0)
    for D, _ in (oracle.fw_naive(W), oracle.fw_blocked(W, 4)):
        assert (np.diag(D) == 0).all()


def test_single_vertex_and_empty_graph():
    D, P = oracle.fw_blocked(np.zeros((1, 1), np.float32), 64)
    assert D[0, 0] == 0 and P[0, 0] == -1
    W = np.full((5, 5), INF, dtype=np.float32)
    D, P = oracle.fw_blocked(W, 2)
    expect = np.full((5, 5), INF, dtype=np.float32)
    np.fill_diagonal(expect, 0)
    np.testing.assert_array_equal(D, expect)
    assert (P == -1).all()


# ---------------------------------------------------------------- special cases of the blocking

@pytest.mark.parametrize("kind", ["int", "real"])
def test_bs1_and_bs_ge_n_reduce_to_naive(kind):
    # With BS=1 every round is one k and the four phases are naive FW's sweep;
    # with BS>=n there is one round whose phase 1 is naive FW (Section 4.1).
    for n, seed in ((17, 1), (40, 2)):
        W = _w(n, seed, 1, 20, density=0.6, kind=kind)
        Dn, Pn = oracle.fw_naive(W)
        for bs in (1, n, n + 5):
            Db, Pb = oracle.fw_blocked(W, bs)
            np.testing.assert_array_equal(Db, Dn)
            np.testing.assert_array_equal(Pb, Pn)


def test_block_size_does_not_change_integer_distances():
    W = _w(100, 3, 1, 1000, density=0.5)
    ref, _ = oracle.fw_naive(W)
    for bs in (2, 7, 16, 32, 64, 99):
        D, P = oracle.fw_blocked(W, bs)
        np.testing.assert_array_equal(D, ref)
        assert oracle.check_paths(W, D, P, all_pairs(100)) == 0


# ---------------------------------------------------------------- library cross-checks

@pytest.mark.parametrize("n,density", [(64, 1.0), (150, 0.3), (257, 0.7)])
def test_scipy_floyd_warshall_int(n, density):
    W = _w(n, n, 1, 1000, density)
    ref = _scipy_apsp(W)
    for D, _ in (oracle.fw_naive(W), oracle.fw_blocked(W, 32)):
        np.testing.assert_array_equal(D.astype(np.float64), ref)


def test_scipy_floyd_warshall_real():
    W = _w(200, 9, kind="real", density=0.8)
    ref = _scipy_apsp(W)
    for D, _ in (oracle.fw_naive(W), oracle.fw_blocked(W, 64)):
        np.testing.assert_allclose(D.astype(np.float64), ref, rtol=1e-5)


def test_dijkstra_and_bellman_ford_vs_scipy():
    W = _w(120, 4, 1, 50, density=0.4)
    G = csg.csgraph_from_dense(W.astype(np.float64), null_value=np.inf)
    ref = csg.dijkstra(G, directed=True)
    for s in (0, 17, 119):
        np.testing.assert_array_equal(oracle.dijkstra(W, s), ref[s])
        np.testing.assert_array_equal(oracle.bellman_ford(W, s), ref[s])


@pytest.mark.parametrize("n,density", [(150, 0.3), (300, 1.0)])
def test_dijkstra_and_bellman_ford_real_weights_vs_scipy(n, density):
    # real weights U(0,1] (the n=32768 real workload's distribution): the oracle's double
    # precision Dijkstra checks sampled rows of that solve at 1e-5, so it is pinned on such
    # graphs too, against scipy's Dijkstra (also double precision) to rounding
    W = _w(n, 7 + n, 0, 1, density=density, kind="real")
    G = csg.csgraph_from_dense(W.astype(np.float64), null_value=np.inf)
    ref = csg.dijkstra(G, directed=True)
    for s in (0, n // 2, n - 1):
        got = oracle.dijkstra(W, s)
        assert (np.isfinite(got) == np.isfinite(ref[s])).all()
        fin = np.isfinite(got)
        np.testing.assert_allclose(got[fin], ref[s][fin], rtol=1e-12, atol=0)
        np.testing.assert_allclose(oracle.bellman_ford(W, s)[fin], ref[s][fin], rtol=1e-12, atol=0)


# ---------------------------------------------------------------- structure of P

def _interior(p):
    return p[1:-1]


@pytest.mark.parametrize("bs", [None, 8])
def test_P_is_last_added_intermediate(bs):
    # Naive FW: the last strict improvement of D[i][j] happens at the largest
    # intermediate vertex of the final path. Blocked FW: it happens in the
    # round of the largest block that holds an interior vertex of the path.
    n = 60
    W = _w(n, 5, 1, 100, density=0.35)
    D, P = oracle.fw_naive(W) if bs is None else oracle.fw_blocked(W, bs)
    for i in range(n):
        for j in range(n):
            if i == j or not np.isfinite(D[i, j]):
                continue
            p = oracle.path(P, i, j)
            inner = _interior(p)
            if not inner:
                assert P[i, j] == -1
            elif bs is None:
                assert P[i, j] == max(inner)
            else:
                assert P[i, j] // bs == max(v // bs for v in inner)


def test_checkers_detect_tampering():
    n = 40
    W = _w(n, 6, 1, 30, density=0.5)
    D, P = oracle.fw_blocked(W, 8)
    pairs = all_pairs(n)
    assert oracle.check_paths(W, D, P, pairs) == 0
    assert oracle.check_invariants(W, D) == 0
    i, j = np.argwhere((P >= 0))[0]
    Dbad = D.copy()
    Dbad[i, j] -= 1
    assert oracle.check_paths(W, Dbad, P, pairs) > 0
    Dbad = D.copy()
    Dbad[i, j] += 1
    assert oracle.check_invariants(W, Dbad) > 0
    Pbad = P.copy()
    Pbad[i, j] = (P[i, j] + 1) % n if (P[i, j] + 1) % n not in (i, j) else (P[i, j] + 2) % n
    assert oracle.check_paths(W, D, Pbad, pairs) > 0
    row = D[3].copy()
    assert oracle.check_bellman_row(W, row) == 0
    row[np.argmax(np.where(np.isfinite(row), row, -1))] += 5
    assert oracle.check_bellman_row(W, row) > 0


def test_paths_and_invariants_real_weights():
    n = 120
    W = _w(n, 8, kind="real", density=0.6)
    D, P = oracle.fw_blocked(W, 16)
    assert oracle.check_paths(W, D, P, random_pairs(n, 3000, 1), rtol=1e-5) == 0
    assert oracle.check_invariants(W, D, rtol=1e-5) == 0


# ---------------------------------------------------------------- planted mistakes

_MUTANTS = {
    "le_instead_of_lt_blocked": ("float c = D[i * n + k] + D[k * n + j];\n        if (c < D[i * n + j]) {\n"
                                 "          D[i * n + j] = c;\n          P[i * n + j] = (int32_t)k;\n        }\n      }\n}\n\n/* Blocked",
                                 "float c = D[i * n + k] + D[k * n + j];\n        if (c <= D[i * n + j]) {\n"
                                 "          D[i * n + j] = c;\n          P[i * n + j] = (int32_t)k;\n        }\n      }\n}\n\n/* Blocked"),
    "transposed_operand": ("static void fw_block", None),
    "local_k_in_P": ("P[i * n + j] = (int32_t)k;\n        }\n      }\n}\n\n/* Blocked",
                     "P[i * n + j] = (int32_t)(k - k0);\n        }\n      }\n}\n\n/* Blocked"),
    "phase3_dropped": ("if (i != r) fw_block(D, P, n, bs, i, r, r);", "(void)0;"),
    "phase4_before_panels": (None, None),
    "diagonal_not_zeroed": ("for (int64_t i = 0; i < n; ++i) D[i * n + i] = 0.0f;", "(void)0;"),
    "naive_wrong_k_column": ("float c = D[i * n + k] + D[k * n + j];\n        if (c < D[i * n + j]) {\n"
                             "          D[i * n + j] = c;\n          P[i * n + j] = (int32_t)k;\n        }\n      }\n}\n\n/* FW_BLOCK",
                             "float c = D[i * n + k] + D[j * n + k];\n        if (c < D[i * n + j]) {\n"
                             "          D[i * n + j] = c;\n          P[i * n + j] = (int32_t)k;\n        }\n      }\n}\n\n/* FW_BLOCK"),
}


def _mutate(src: str, name: str) -> str:
    if name == "transposed_operand":
        # inside FW_BLOCK only: A[i][k] read as A[k][i]
        head, tail = src.split("static void fw_block", 1)
        body, rest = tail.split("/* Blocked", 1)
        assert "D[i * n + k] + D[k * n + j]" in body
        body = body.replace("D[i * n + k] + D[k * n + j]", "D[k * n + i] + D[k * n + j]")
        return head + "static void fw_block" + body + "/* Blocked" + rest
    if name == "phase4_before_panels":
        a = ("    for (int64_t j = 0; j < R; ++j)\n      if (j != r) fw_block(D, P, n, bs, r, j, r);                    /* phase 2 */\n"
             "    for (int64_t i = 0; i < R; ++i)\n      if (i != r) fw_block(D, P, n, bs, i, r, r);                    /* phase 3 */\n")
        b = ("    for (int64_t i = 0; i < R; ++i)\n      if (i != r)\n        for (int64_t j = 0; j < R; ++j)\n"
             "          if (j != r) fw_block(D, P, n, bs, i, j, r);                /* phase 4 */\n")
        assert a in src and b in src
        return src.replace(a, "@@A@@").replace(b, a).replace("@@A@@", b)
    old, new = _MUTANTS[name]
    assert src.count(old) == 1, name
    return src.replace(old, new)


def _build_mutant(tmp_path, name):
    here = os.path.dirname(oracle.__file__)
    src = open(os.path.join(here, "apsp_oracle.c")).read()
    d = tmp_path / name
    d.mkdir()
    (d / "apsp_oracle.c").write_text(_mutate(src, name))
    shutil.copy(os.path.join(here, "apsp_oracle.h"), d / "apsp_oracle.h")
    so = d / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                    str(d / "apsp_oracle.c"), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    f32p, i32p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
    lib.oracle_fw_naive.argtypes = [f32p, ctypes.c_int, f32p, i32p]
    lib.oracle_fw_blocked.argtypes = [f32p, ctypes.c_int, ctypes.c_int, f32p, i32p]
    return lib


def _run(lib, W, bs):
    W = np.ascontiguousarray(W, dtype=np.float32)
    n = W.shape[0]
    D = np.empty_like(W)
    P = np.empty((n, n), np.int32)
    f32p, i32p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
    if bs is None:
        lib.oracle_fw_naive(W.ctypes.data_as(f32p), n, D.ctypes.data_as(f32p), P.ctypes.data_as(i32p))
    else:
        lib.oracle_fw_blocked(W.ctypes.data_as(f32p), n, bs, D.ctypes.data_as(f32p), P.ctypes.data_as(i32p))
    return D, P


def _pins_pass(lib) -> bool:
    """The oracle pins above, re-run against a candidate build."""
    for name in ("tie_break_4.txt", "blocked_vs_naive_4.txt"):
        g = load_golden(name)
        for bs, dk, pk in ((None, "D_naive", "P_naive"), (g["bs"], "D_blocked", "P_blocked")):
            D, P = _run(lib, g["W"], bs)
            if not (np.array_equal(D, g[dk]) and np.array_equal(P, g[pk])):
                return False
    for seed in range(3):
        W = _w(7, 300 + seed, 1, 9, 0.5)
        np.fill_diagonal(W, 4.0)
        ref = brute_force_apsp(W)
        for bs in (None, 2, 3):
            D, P = _run(lib, W, bs)
            if not np.array_equal(D.astype(np.float64), ref):
                return False
            if oracle.check_paths(W, D, P, all_pairs(7)) != 0:
                return False
    return True


def test_pins_accept_the_real_oracle(tmp_path):
    lib = ctypes.CDLL(oracle.build())
    f32p, i32p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
    lib.oracle_fw_naive.argtypes = [f32p, ctypes.c_int, f32p, i32p]
    lib.oracle_fw_blocked.argtypes = [f32p, ctypes.c_int, ctypes.c_int, f32p, i32p]
    assert _pins_pass(lib)


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
@pytest.mark.parametrize("name", sorted(_MUTANTS))
def test_pins_reject_planted_mistake(tmp_path, name):
    assert not _pins_pass(_build_mutant(tmp_path, name))
