"""The paper's blocked design on the host cores (the parallel CPU baseline) equals the serial
blocked oracle bit for bit: same candidates, same order, same fp32 additions."""

import numpy as np
import pytest

import oracle
from oracle import host_blocked
from paper_1811_01201_gb300 import inputs


@pytest.mark.parametrize("n,bs", [(1, 16), (5, 16), (64, 16), (65, 16), (130, 32), (200, 64), (257, 64), (100, 128)])
@pytest.mark.parametrize("kind", ["int", "real"])
def test_equals_blocked_oracle(n, bs, kind):
    W = inputs.dense_digraph(n, 40 + n, 0 if kind == "real" else 1, 1 if kind == "real" else 50,
                             density=0.6, kind=kind).numpy()
    D, P = host_blocked.fw_blocked(W, bs)
    Dr, Pr = oracle.fw_blocked(W, bs)
    np.testing.assert_array_equal(D, Dr)
    np.testing.assert_array_equal(P, Pr)


def test_ties_keep_the_earlier_k():
    # complete graph with unit weights: every two-hop path ties with the direct edge
    n = 70
    W = np.ones((n, n), dtype=np.float32)
    D, P = host_blocked.fw_blocked(W, 16)
    assert (P == -1).all()
    assert (D[~np.eye(n, dtype=bool)] == 1.0).all()


def test_reports_its_thread_count():
    assert host_blocked.threads() >= 1


@pytest.mark.parametrize("n,bs,lo,hi,density,kind", [
    (1024, 64, 1, 1000, 0.5, "int"),    # the shape of the n = 8192 density-0.5 workload
    (1024, 128, 1, 1000, 1.0, "int"),
    (768, 64, 0, 1, 1.0, "real"),
    (640, 128, 1, 15, 0.3, "int"),      # a 16-bit-eligible graph whose elements improve
])
def test_equals_blocked_oracle_at_larger_sizes(n, bs, lo, hi, density, kind):
    # the whole-matrix GPU parity tests at the benchmark sizes take this implementation as the
    # oracle (the serial one needs minutes there), so it is pinned here at sizes that span many
    # blocks of every phase, with the workloads' weight distributions
    W = inputs.dense_digraph(n, 7 * n + bs, lo, hi, density=density, kind=kind).numpy()
    D, P = host_blocked.fw_blocked(W, bs)
    Dr, Pr = oracle.fw_blocked(W, bs)
    np.testing.assert_array_equal(D, Dr)
    np.testing.assert_array_equal(P, Pr)
