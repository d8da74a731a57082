"""GPU parity of the persistent batched launch (apsp_fw_batched / apsp_batch_*).

Every graph of a batch must equal oracle.fw_blocked(W, 32) bit for bit and
the single-graph path with BS = 32, whichever order the persistent CTAs take
the graphs in.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01201_gb300 as apsp
from paper_1811_01201_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _make(ns, seed, lo=1, hi=100, density=0.7, kind="int"):
    Ws = [inputs.dense_digraph(n, inputs.batch_graph_seed(seed, g), lo, hi, density=density, kind=kind)
          for g, n in enumerate(ns)]
    Wd = [w.to(DEV) for w in Ws]
    Dd = [torch.empty_like(w) for w in Wd]
    Pd = [torch.empty(w.shape, dtype=torch.int32, device=DEV) for w in Wd]
    return Ws, Wd, Dd, Pd


def _check_all(Ws, Dd, Pd, bs=32):
    torch.cuda.synchronize()
    for g, W in enumerate(Ws):
        Dr, Pr = oracle.fw_blocked(W.numpy(), bs)
        np.testing.assert_array_equal(Dd[g].cpu().numpy(), Dr, err_msg=f"graph {g} n={W.shape[0]}")
        np.testing.assert_array_equal(Pd[g].cpu().numpy(), Pr, err_msg=f"graph {g} n={W.shape[0]}")


def test_log_uniform_batch_int():
    ns = inputs.batch_sizes(160, seed=6)
    Ws, Wd, Dd, Pd = _make(ns, 6)
    bs = apsp.apsp_fw_batched(Wd, Dd, Pd)
    assert all(b == 32 for b in bs)
    _check_all(Ws, Dd, Pd)


def test_edge_orders():
    ns = [1, 2, 3, 16, 31, 32, 33, 63, 64, 65, 96, 127, 128, 129, 255, 256, 257, 500, 511, 512]
    Ws, Wd, Dd, Pd = _make(ns, 17, density=0.5)
    apsp.apsp_fw_batched(Wd, Dd, Pd)
    _check_all(Ws, Dd, Pd)


def test_real_weights_and_large_integers_use_generic_path():
    ns = [40, 100, 200, 333, 512]
    Ws, Wd, Dd, Pd = _make(ns, 8, kind="real", density=0.8)
    apsp.apsp_fw_batched(Wd, Dd, Pd)
    _check_all(Ws, Dd, Pd)
    Ws, Wd, Dd, Pd = _make(ns, 9, lo=1, hi=1_000_000, density=0.3)
    apsp.apsp_fw_batched(Wd, Dd, Pd)
    _check_all(Ws, Dd, Pd)


def test_batched_equals_single_graph_path():
    ns = [50, 130, 260, 400]
    Ws, Wd, Dd, Pd = _make(ns, 10, lo=1, hi=1000, density=0.6)
    apsp.apsp_fw_batched(Wd, Dd, Pd)
    torch.cuda.synchronize()
    for g, n in enumerate(ns):
        D1 = torch.empty_like(Wd[g])
        P1 = torch.empty_like(Pd[g])
        apsp.apsp_fw_ex(Wd[g], D1, P1, bs=32, dtype=apsp.DTYPE_F32)
        torch.cuda.synchronize()
        assert torch.equal(D1, Dd[g]) and torch.equal(P1, Pd[g])


def test_in_place_batch():
    ns = [70, 300]
    Ws, Wd, Dd, Pd = _make(ns, 11)
    apsp.apsp_fw_batched(Wd, Wd, Pd)  # W aliases D
    _check_all(Ws, Wd, Pd)


def test_reusable_batch_in_cuda_graph():
    ns = inputs.batch_sizes(64, seed=12)
    Ws, Wd, Dd, Pd = _make(ns, 12)
    b = apsp.Batch(Wd, Dd, Pd)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        b.launch(stream=s)  # warm-up outside capture
    s.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.launch(stream=s)
    for Dx in Dd:
        Dx.fill_(-5.0)
    for Px in Pd:
        Px.fill_(7)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    _check_all(Ws, Dd, Pd)
    b.close()


def test_autotuned_tiles_give_identical_results():
    # graphs in every size class; the autotuner runs each tile height, then the batch is
    # relaunched with the chosen ones: all results equal the oracle with BS = 32
    ns = [20, 50, 64, 65, 100, 128, 129, 200, 256, 257, 400, 512]
    Ws, Wd, Dd, Pd = _make(ns, 15, density=0.6)
    b = apsp.Batch(Wd, Dd, Pd)
    rows = b.autotune()
    assert len(rows) == 4 and all(r in (0, 32, 64, 128) for r in rows)  # 0: the per-graph size rule
    for Dx in Dd:
        Dx.fill_(-3.0)
    b.launch()
    _check_all(Ws, Dd, Pd)
    b.close()
    # classes without graphs report -1; in-place batches cannot be autotuned
    Ws, Wd, Dd, Pd = _make([30, 40], 16)
    b = apsp.Batch(Wd, Dd, Pd)
    rows = b.autotune()  # the choice follows timings, so a second run may pick another tile
    assert rows[1:] == [-1, -1, -1] and rows[0] in (0, 32, 64, 128)
    b.launch()
    _check_all(Ws, Dd, Pd)
    b.close()
    b = apsp.Batch(Wd, Wd, Pd)
    with pytest.raises(apsp.ApspError) as e:
        b.autotune()
    assert e.value.status == apsp.APSP_EINVAL
    b.close()


def test_invalid_batches_rejected():
    Ws, Wd, Dd, Pd = _make([40, 50], 13)
    Wd[1][3, 4] = -2.0
    with pytest.raises(apsp.ApspError) as e:
        apsp.apsp_fw_batched(Wd, Dd, Pd)
    assert e.value.status == apsp.APSP_EINVAL
    big = torch.zeros((513, 513), device=DEV)
    with pytest.raises(apsp.ApspError) as e:
        apsp.apsp_fw_batched([big], [big.clone()], [torch.zeros((513, 513), dtype=torch.int32, device=DEV)])
    assert e.value.status == apsp.APSP_EINVAL
    with pytest.raises(apsp.ApspError) as e:
        apsp.apsp_fw_batched(Wd[:1], Dd[:1], Pd[:1], bs=64)
    assert e.value.status == apsp.APSP_EINVAL
    # the context is still usable
    Ws, Wd, Dd, Pd = _make([45], 14)
    apsp.apsp_fw_batched(Wd, Dd, Pd)
    _check_all(Ws, Dd, Pd)


def test_full_size_batch_in_cuda_graph_sampled():
    # the benchmark's batch (4096 graphs, n log-uniform in [16,512], U[1,100], density 0.7) run as
    # one CUDA-graph-replayed persistent launch; 48 sampled graphs checked against the oracle
    count, seed = 4096, 6
    ns = inputs.batch_sizes(count, seed)
    Wd = [inputs.dense_digraph(n, inputs.batch_graph_seed(seed, g), 1, 100, density=0.7, device=DEV)
          for g, n in enumerate(ns)]
    Dd = [torch.empty_like(w) for w in Wd]
    Pd = [torch.empty(w.shape, dtype=torch.int32, device=DEV) for w in Wd]
    b = apsp.Batch(Wd, Dd, Pd)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        b.launch(stream=s)
    graph.replay()
    torch.cuda.synchronize()
    rng = np.random.default_rng(0)
    sample = list(rng.choice(count, size=44, replace=False)) + [int(np.argmax(ns)), int(np.argmin(ns))]
    for g in sample:
        Dr, Pr = oracle.fw_blocked(Wd[g].cpu().numpy(), 32)
        np.testing.assert_array_equal(Dd[g].cpu().numpy(), Dr)
        np.testing.assert_array_equal(Pd[g].cpu().numpy(), Pr)
    b.close()
