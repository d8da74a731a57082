"""Whole-matrix parity at the benchmark sizes: every element of D and P from the GPU
against the blocked oracle with the same block size (Section 4.1's phase order, Section
3's P as the most recently added intermediate, strict '<' per Section 4.2).

The serial oracle needs minutes to hours at these orders, so the reference here is
oracle/host_blocked.c: the same blocked sweep on the host cores (OpenMP over the blocks
of each phase), pinned bit for bit to the serial oracle by tests/test_host_blocked.py.
Both sides perform the same fp32 additions in the same per-element order, so D and P
must match exactly, for integer and for real weights alike.

At n = 8192 and above the phase-3 grid has many waves, so these runs cover what the
small-n tests cannot: the staggered second half of the first wave, element offsets of
a 2^26- and 2^30-element matrix, and the sparse late-round P writes of a multi-wave grid.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01201_gb300 as apsp
from oracle import host_blocked
from paper_1811_01201_gb300 import inputs
from tests.helpers import random_pairs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _solve(n, seed, lo, hi, density, kind, bs, dtype):
    Wd = inputs.dense_digraph(n, seed, lo, hi, density=density, kind=kind, device=DEV)
    D = torch.empty_like(Wd)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    info = apsp.apsp_fw_ex(Wd, D, P, bs=bs, dtype=dtype)
    torch.cuda.synchronize()
    W = Wd.cpu().numpy()
    del Wd
    Dh, Ph = D.cpu().numpy(), P.cpu().numpy()
    del D, P
    torch.cuda.empty_cache()
    return W, Dh, Ph, info


def _assert_equal(name, got, want):
    if np.array_equal(got, want):
        return
    bad = np.argwhere(got != want)
    i, j = (int(x) for x in bad[0])
    raise AssertionError(f"{name}: {len(bad)} elements differ; first at ({i}, {j}): got {got[i, j]}, "
                         f"oracle {want[i, j]}")


def _whole_matrix(W, D, P, bs):
    Dr, Pr = host_blocked.fw_blocked(W, bs)
    _assert_equal("D", D, Dr)
    _assert_equal("P", P, Pr)


@pytest.mark.parametrize("bs", [64, 128])
def test_n8192_int_density_half(bs):
    # the n = 8192 workload: integer weights U[1,1000], each edge present with probability 0.5
    W, D, P, info = _solve(8192, 2, 1, 1000, 0.5, "int", bs, apsp.DTYPE_F32)
    assert info.bs_used == bs and info.dtype_used == apsp.DTYPE_F32
    _whole_matrix(W, D, P, bs)


def test_n8192_real_weights():
    # real weights U(0,1]: the tag kernel of phase 3 and the plain-compare phases 1-2
    W, D, P, info = _solve(8192, 4, 0, 1, 1.0, "real", 64, apsp.DTYPE_F32)
    assert info.dtype_used == apsp.DTYPE_F32
    _whole_matrix(W, D, P, 64)


@pytest.mark.parametrize("bs", [64, 128])
def test_u16_path_on_a_graph_that_improves(bs):
    # 16-bit eligible (15 * 4095 = 61425 < 65535) with absent edges, so that many elements
    # improve in every round and the 16-bit path's P search runs
    W, D, P, info = _solve(4096, 8, 1, 15, 0.3, "int", bs, apsp.DTYPE_AUTO)
    assert info.dtype_used == apsp.DTYPE_U16X2 and info.bs_used == bs
    _whole_matrix(W, D, P, bs)
    improved = int((P >= 0).sum())
    assert improved > 4096 * 4096 // 4  # the run did real work in phase 3


@pytest.mark.slow
def test_n32768_int_whole_matrix_and_a_million_walks():
    # the headline workload: n = 32768, dense, integer weights U[1,1000], BS = 64
    n, bs = 32768, 64
    W, D, P, info = _solve(n, 3, 1, 1000, 1.0, "int", bs, apsp.DTYPE_F32)
    assert info.bs_used == bs and info.dtype_used == apsp.DTYPE_F32
    pairs = random_pairs(n, 1_000_000, 17)
    assert oracle.check_paths(W, D, P, pairs) == 0
    _whole_matrix(W, D, P, bs)


@pytest.mark.slow
def test_u16_benchmark_workload_whole_matrix():
    # the benchmark's 16-bit workload on which elements improve: n = 16384, U[1,3], half the edges
    # present (3 * 16383 < 65535), at the library's default block size
    W, D, P, info = _solve(16384, 9, 1, 3, 0.5, "int", 0, apsp.DTYPE_AUTO)
    assert info.dtype_used == apsp.DTYPE_U16X2
    _whole_matrix(W, D, P, info.bs_used)
