"""The seeded input generator: published SplitMix64 values, slab independence, ranges."""

import math

import numpy as np
import torch

from paper_1811_01201_gb300 import inputs


def test_splitmix64_published_first_output():
    # SplitMix64 seeded with 0 returns 0xE220A8397B1DCDAF first (state += gamma, then mix)
    assert inputs.mix64_int(inputs._GAMMA) == 0xE220A8397B1DCDAF
    z = inputs.mix64(torch.tensor([inputs._signed(inputs._GAMMA)], dtype=torch.int64))
    assert int(z) & inputs._MASK64 == 0xE220A8397B1DCDAF


def test_tensor_mix_matches_python_ints():
    xs = [0, 1, 12345, 2**40 + 7, 2**63 - 1, 2**63, 2**64 - 1]
    t = torch.tensor([inputs._signed(x) for x in xs], dtype=torch.int64)
    got = [int(v) & inputs._MASK64 for v in inputs.mix64(t)]
    assert got == [inputs.mix64_int(x) for x in xs]


def test_rows_and_slabs_are_consistent():
    full = inputs.dense_digraph(300, 11, 1, 1000, density=0.5, slab=64)
    part = inputs.dense_digraph(300, 11, 1, 1000, density=0.5, rows=(123, 200), slab=7)
    assert torch.equal(full[123:200], part)


def test_value_ranges():
    W = inputs.dense_digraph(400, 2, 1, 1000, density=0.5).numpy()
    off = ~np.eye(400, dtype=bool)
    fin = np.isfinite(W) & off
    assert (np.diag(W) == 0).all()
    assert abs(fin.sum() / off.sum() - 0.5) < 0.02
    assert W[fin].min() == 1 and W[fin].max() == 1000
    assert (W[fin] == np.round(W[fin])).all()
    R = inputs.dense_digraph(300, 4, kind="real").numpy()
    v = R[~np.eye(300, dtype=bool)]
    assert v.min() > 0 and v.max() <= 1 and np.isfinite(v).all()


def test_batch_and_request_generators():
    ns = inputs.batch_sizes(4096, 6)
    assert min(ns) >= 16 and max(ns) <= 512
    med = np.median(ns)
    assert abs(math.log(med) - (math.log(16) + math.log(512)) / 2) < 0.15
    ls = inputs.lognormal_sizes(2000, 7)
    assert 32 <= min(ls) and max(ls) <= 4096 and abs(np.median(ls) - 256) < 30
    t = inputs.poisson_arrivals(5000, 7, 200.0)
    gaps = np.diff([0.0] + t)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0
