"""GPU tests of the continuous-batching server (apsp_serve_*).

Each served result must equal the same graph solved alone with apsp_fw's
default options (and the oracle with the reported block size), whatever else
shares the GPU; admission must respect the HBM budget; failures are reported
as status codes.
"""

import threading
import time

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01201_gb300 as apsp
from paper_1811_01201_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _graphs(count, seed, n_hi=1024):
    ns = inputs.lognormal_sizes(count, seed, median=180, sigma=0.8, n_lo=32, n_hi=n_hi)
    return [inputs.dense_digraph(n, inputs.batch_graph_seed(seed, g), 1, 64).numpy() for g, n in enumerate(ns)]


def _alone(W):
    n = W.shape[0]
    Wd = torch.from_numpy(W).to(DEV)
    D = torch.empty_like(Wd)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw(Wd, D, P)
    torch.cuda.synchronize()
    return D.cpu().numpy(), P.cpu().numpy()


def test_mixed_stream_matches_alone_and_oracle():
    Ws = _graphs(48, 21)
    Ws.append(inputs.dense_digraph(1500, 99, 1, 64).numpy())  # one graph above the batched limit
    with apsp.Server(4 << 30, max_slots=32) as srv:
        ids = [srv.submit(W) for W in Ws]
        results = [srv.poll(j, W.shape[0], timeout_ms=60000) for j, W in zip(ids, Ws)]
        st = srv.stats()
    assert st.completed == len(Ws) and st.rejected == 0
    assert 0 < st.p50_ms <= st.p99_ms <= st.max_ms
    for W, (D, P, bs) in zip(Ws, results):
        Da, Pa = _alone(W)
        np.testing.assert_array_equal(D, Da)
        np.testing.assert_array_equal(P, Pa)
        if W.shape[0] <= 600:
            Dr, Pr = oracle.fw_blocked(W, bs)
            np.testing.assert_array_equal(D, Dr)
            np.testing.assert_array_equal(P, Pr)


def test_poll_into_reused_buffers():
    Ws = _graphs(12, 24)
    bufD = np.empty(1024 * 1024, np.float32)
    bufP = np.empty(1024 * 1024, np.int32)
    with apsp.Server(2 << 30, max_slots=8) as srv:
        ids = [srv.submit(W) for W in Ws]
        for j, W in zip(ids, Ws):
            n = W.shape[0]
            D, P, bs = srv.poll(j, n, timeout_ms=60000, out=(bufD[:n * n].reshape(n, n), bufP[:n * n].reshape(n, n)))
            assert np.shares_memory(D, bufD) and np.shares_memory(P, bufP)
            Dr, Pr = oracle.fw_blocked(W, bs)
            np.testing.assert_array_equal(D, Dr)
            np.testing.assert_array_equal(P, Pr)
        with pytest.raises(ValueError):
            srv.poll(srv.submit(Ws[0]), Ws[0].shape[0], out=(bufD[:10], bufP[:10]))


def test_concurrent_submitters_and_overlap():
    Ws = _graphs(60, 22, n_hi=512)
    out = {}
    with apsp.Server(2 << 30, max_slots=64) as srv:
        def worker(lo, hi):
            for g in range(lo, hi):
                out[g] = (srv.submit(Ws[g]), Ws[g].shape[0])
                time.sleep(0.001)
        th = [threading.Thread(target=worker, args=(k * 15, (k + 1) * 15)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for g in range(len(Ws)):
            jid, n = out[g]
            D, P, _ = srv.poll(jid, n, timeout_ms=60000)
            Da, Pa = _alone(Ws[g])
            assert np.array_equal(D, Da) and np.array_equal(P, Pa)


def test_budget_admission_and_rejection():
    Ws = _graphs(12, 23, n_hi=512)
    n_big = max(W.shape[0] for W in Ws)
    budget = 8 * n_big * n_big + 64 * 1024  # room for about one largest job at a time
    with apsp.Server(max(budget, 1 << 20), max_slots=8) as srv:
        ids = [srv.submit(W) for W in Ws]
        for j, W in zip(ids, Ws):
            D, P, _ = srv.poll(j, W.shape[0], timeout_ms=60000)
            Da, Pa = _alone(W)
            assert np.array_equal(D, Da) and np.array_equal(P, Pa)
        st = srv.stats()
        assert st.hbm_peak <= max(budget, 1 << 20)
        # a job that can never fit is refused at submit
        with pytest.raises(apsp.ApspError) as e:
            srv.submit(np.zeros((1024, 1024), np.float32))
        assert e.value.status == apsp.APSP_ENOMEM


def test_failures_are_status_codes():
    with apsp.Server(1 << 30, max_slots=4) as srv:
        bad = np.ones((40, 40), np.float32)
        bad[1, 2] = -1
        with pytest.raises(apsp.ApspError) as e:
            srv.submit(bad)
        assert e.value.status == apsp.APSP_EINVAL
        bad[1, 2] = np.nan
        with pytest.raises(apsp.ApspError) as e:
            srv.submit(bad)
        assert e.value.status == apsp.APSP_EINVAL
        with pytest.raises(apsp.ApspError) as e:
            srv.poll(123456, 10, timeout_ms=0)
        assert e.value.status == apsp.APSP_ENOTFOUND
        jid = srv.submit(_graphs(1, 24)[0])
        r = srv.try_poll(jid, 1, timeout_ms=0, want_result=False)  # may or may not be ready
        if r is None:
            srv.poll(jid, 1, timeout_ms=60000, want_result=False)
        assert srv.stats().rejected == 2


def test_destroy_with_pending_work():
    Ws = _graphs(30, 25, n_hi=512)
    srv = apsp.Server(1 << 30, max_slots=2)
    for W in Ws:
        srv.submit(W)
    srv.close()  # cancels queued jobs, drains the device, joins the scheduler
    # a fresh server still works afterwards
    with apsp.Server(1 << 30, max_slots=2) as srv2:
        j = srv2.submit(Ws[0])
        D, P, _ = srv2.poll(j, Ws[0].shape[0], timeout_ms=60000)
        Da, Pa = _alone(Ws[0])
        assert np.array_equal(D, Da) and np.array_equal(P, Pa)
