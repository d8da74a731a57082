"""GPU parity of the batched device path walk (apsp_paths).

Every walk must give the vertex list (or the failure) of oracle.path on a host
copy of the same P with the same capacity, and on solved graphs the walks must
be simple paths of weight D[i][j] (oracle.check_paths).
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01201_gb300 as apsp
from paper_1811_01201_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _walk(P_dev, pairs, cap):
    out, lens = apsp.apsp_paths(P_dev, torch.from_numpy(pairs).to(DEV), cap)
    torch.cuda.synchronize()
    return out.cpu().numpy(), lens.cpu().numpy()


def _compare(P_host, pairs, out, lens, cap):
    for t, (i, j) in enumerate(pairs):
        ref = oracle.path(P_host, int(i), int(j), cap)
        if ref is None:
            assert lens[t] == -1, (t, i, j, lens[t])
        else:
            assert lens[t] == len(ref), (t, i, j, lens[t], ref)
            assert list(out[t, :lens[t]]) == ref, (t, i, j)


def _solve(n, seed, lo, hi, density=1.0, kind="int", bs=0):
    W = inputs.dense_digraph(n, seed, lo, hi, density=density, kind=kind, device=DEV)
    D = torch.empty_like(W)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw_ex(W, D, P, bs=bs)
    torch.cuda.synchronize()
    return W, D, P


def test_all_pairs_of_a_solved_graph():
    n = 150
    W, D, P = _solve(n, 21, 1, 100, density=0.2)
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pairs = np.stack([ii.ravel(), jj.ravel()], 1).astype(np.int32)
    out, lens = _walk(P, pairs, n)
    Ph = P.cpu().numpy()
    _compare(Ph, pairs, out, lens, n)
    assert oracle.check_paths(W.cpu().numpy(), D.cpu().numpy(), Ph, pairs[pairs[:, 0] != pairs[:, 1]]) == 0


def test_real_weights_and_small_capacities():
    n = 300
    W, D, P = _solve(n, 22, 0, 1, kind="real")
    pairs = inputs.vertex_pairs(4000, n, 5).numpy()
    Ph = P.cpu().numpy()
    for cap in (1, 2, 3, 4, 8, 300, 1000):
        out, lens = _walk(P, pairs, cap)
        _compare(Ph, pairs, out, lens, cap)
    out, lens = _walk(P, pairs, n)
    ok = pairs[:, 0] != pairs[:, 1]
    assert oracle.check_paths(W.cpu().numpy(), D.cpu().numpy(), Ph, pairs[ok], rtol=1e-5) == 0


def test_malformed_matrices_fail_exactly_where_the_oracle_does():
    rng = np.random.default_rng(3)
    for trial in range(12):
        n = int(rng.integers(2, 40))
        Ph = rng.integers(-1, n, size=(n, n)).astype(np.int32)
        if trial % 2:
            Ph[rng.random((n, n)) < 0.7] = -1
        P = torch.from_numpy(Ph).to(DEV)
        ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        pairs = np.stack([ii.ravel(), jj.ravel()], 1).astype(np.int32)
        for cap in (1, 2, 5, n, 3 * n):
            out, lens = _walk(P, pairs, cap)
            _compare(Ph, pairs, out, lens, cap)


def test_out_of_range_pairs_and_empty_batch():
    n = 40
    _, _, P = _solve(n, 23, 1, 9)
    pairs = np.array([[-1, 3], [3, -1], [n, 0], [0, n], [5, 5], [0, 39]], dtype=np.int32)
    out, lens = _walk(P, pairs, 16)
    assert list(lens[:4]) == [-1, -1, -1, -1]
    assert lens[4] == 1 and out[4, 0] == 5
    assert lens[5] >= 2 and out[5, 0] == 0 and out[5, lens[5] - 1] == 39
    e_out, e_lens = apsp.apsp_paths(P, torch.empty((0, 2), dtype=torch.int32, device=DEV), 8)
    torch.cuda.synchronize()
    assert e_out.numel() == 0 and e_lens.numel() == 0


def test_walks_capture_into_a_cuda_graph():
    n = 200
    _, _, P = _solve(n, 24, 1, 1000, density=0.1)
    pairs = inputs.vertex_pairs(5000, n, 6, device=DEV)
    out = torch.empty((5000, 32), dtype=torch.int32, device=DEV)
    lens = torch.empty((5000,), dtype=torch.int32, device=DEV)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        apsp.apsp_paths(P, pairs, 32, out, lens, stream=s)
    lens.fill_(-7)
    g.replay()
    torch.cuda.synchronize()
    _compare(P.cpu().numpy(), pairs.cpu().numpy(), out.cpu().numpy(), lens.cpu().numpy(), 32)


@pytest.mark.slow
def test_full_size_walks_sampled():
    # the benchmark's walk: 2^20 seeded pairs on the solved n=32768 integer graph (U[1,1000],
    # dense, BS=64), cap 64; 3000 sampled walks against the oracle walk on the host copy of P,
    # and every walk ends at its target
    n, count = 32768, 1 << 20
    _, _, P = _solve(n, 3, 1, 1000, bs=64)
    pairs = inputs.vertex_pairs(count, n, 11, device=DEV)
    out, lens = apsp.apsp_paths(P, pairs, 64)
    torch.cuda.synchronize()
    lens_h = lens.cpu().numpy()
    pairs_h = pairs.cpu().numpy()
    off = pairs_h[:, 0] != pairs_h[:, 1]
    assert (lens_h[off] >= 2).all() and (lens_h[~off] == 1).all()
    L = torch.from_numpy(lens_h).to(DEV).long()
    last = out.gather(1, (L - 1).clamp_(min=0).view(-1, 1)).view(-1).cpu().numpy()
    assert (last == pairs_h[:, 1]).all()
    Ph = P.cpu().numpy()
    rng = np.random.default_rng(0)
    sample = rng.choice(count, size=3000, replace=False)
    out_s = out[torch.from_numpy(sample).to(DEV)].cpu().numpy()
    _compare(Ph, pairs_h[sample], out_s, lens_h[sample], 64)
