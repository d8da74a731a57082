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


def test_small_jobs_finish_while_an_earlier_large_job_is_on_the_device():
    # Continuous batching: a request that arrives while a large solve runs is admitted, runs
    # beside it and completes first. The large job (n = 12288, fp32 path, about 0.15 s of device
    # work) is submitted first; once its kernels run, small graphs arrive and must all be done
    # while the large one is still in flight. A server that ran jobs one at a time would finish
    # the large job first.
    big = inputs.dense_digraph(12288, 61, 1, 1000, density=0.95).numpy()
    smalls = _graphs(8, 62, n_hi=256)
    with apsp.Server(8 << 30, max_slots=16) as srv:
        jb = srv.submit(big)
        time.sleep(0.03)  # past the large job's host-to-device copy: its rounds are running
        ids = [srv.submit(W) for W in smalls]
        small_results = [srv.poll(j, W.shape[0], timeout_ms=60000) for j, W in zip(ids, smalls)]
        assert srv.try_poll(jb, big.shape[0], timeout_ms=0, want_result=False) is None, \
            "the large job finished before the small jobs that arrived after it"
        D, P, bs = srv.poll(jb, big.shape[0], timeout_ms=120000)
    for W, (Ds, Ps, _) in zip(smalls, small_results):
        Da, Pa = _alone(W)
        assert np.array_equal(Ds, Da) and np.array_equal(Ps, Pa)
    Da, Pa = _alone(big)
    assert np.array_equal(D, Da) and np.array_equal(P, Pa)


def test_a_served_job_whose_device_wait_expires_fails_alone():
    # Failure detection without a GPU fault: the test flag makes the job's bounded device waits
    # expire (its kernels copy no panel slices; 20 ms per CTA wave), so its solve is invalid. The
    # server reads that job's own fault word and fails it with APSP_ETIMEOUT; jobs running beside
    # it return correct results, and the server keeps working.
    bad = inputs.dense_digraph(640, 71, 1, 64).numpy()    # 16-bit path, 10 rounds of BS = 64
    good = inputs.dense_digraph(700, 72, 1, 1000).numpy()  # fp32 path
    smalls = _graphs(6, 73, n_hi=256)
    try:
        with apsp.Server(4 << 30, max_slots=16) as srv:
            jbad = srv.submit(bad, flags=apsp.FLAG_TEST_PANEL_TIMEOUT)
            jgood = srv.submit(good)
            ids = [srv.submit(W) for W in smalls]
            with pytest.raises(apsp.ApspError) as e:
                srv.poll(jbad, bad.shape[0], timeout_ms=60000)
            assert e.value.status == apsp.APSP_ETIMEOUT
            D, P, _ = srv.poll(jgood, good.shape[0], timeout_ms=60000)
            Da, Pa = _alone(good)
            assert np.array_equal(D, Da) and np.array_equal(P, Pa)
            for j, W in zip(ids, smalls):
                Ds, Ps, _ = srv.poll(j, W.shape[0], timeout_ms=60000)
                Da, Pa = _alone(W)
                assert np.array_equal(Ds, Da) and np.array_equal(Ps, Pa)
            # the same graph without the flag is served correctly afterwards
            D, P, bs = srv.poll(srv.submit(bad), bad.shape[0], timeout_ms=60000)
            Da, Pa = _alone(bad)
            assert np.array_equal(D, Da) and np.array_equal(P, Pa)
            st = srv.stats()
            assert st.completed == len(smalls) + 2  # the failed job is not counted as completed
    finally:
        apsp.apsp_device_status(clear=True)  # the device-wide word saw the expired waits too


def test_submit_with_options():
    W = inputs.dense_digraph(300, 74, 1, 30).numpy()  # 16-bit eligible
    with apsp.Server(1 << 30, max_slots=4) as srv:
        for bs, dtype in ((64, apsp.DTYPE_F32), (128, apsp.DTYPE_U16X2), (32, None)):
            D, P, bs_used = srv.poll(srv.submit(W, bs=bs, dtype=dtype), 300, timeout_ms=60000)
            assert bs_used == bs
            Dr, Pr = oracle.fw_blocked(W, bs)
            np.testing.assert_array_equal(D, Dr)
            np.testing.assert_array_equal(P, Pr)
        with pytest.raises(apsp.ApspError) as e:
            srv.submit(W, bs=48)
        assert e.value.status == apsp.APSP_EINVAL
        with pytest.raises(apsp.ApspError) as e:
            srv.submit(W, flags=apsp.FLAG_TIME_PHASES)
        assert e.value.status == apsp.APSP_EINVAL
        with pytest.raises(apsp.ApspError) as e:
            srv.submit(inputs.dense_digraph(300, 75, 1, 1000, density=0.9).numpy(), dtype=apsp.DTYPE_U16X2)
        assert e.value.status == apsp.APSP_EINVAL
