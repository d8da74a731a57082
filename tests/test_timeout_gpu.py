"""Failure detection without a GPU fault: the phase-3 CTAs wait for their panel slices with a
time bound. With the test flag they announce the slices but never copy them, so every wait
expires (20 ms per CTA wave, no copy in flight); the CTAs leave their tiles, set the device
fault word, and the host reads APSP_ETIMEOUT. The context stays usable afterwards."""

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01201_gb300 as apsp
from paper_1811_01201_gb300 import inputs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("kind", ["int", "real"])
def test_expired_panel_wait_is_reported_and_the_context_survives(kind):
    n = 256  # 2 x 2 tiles, 4 rounds of BS = 64: each phase-3 launch is one wave
    W = inputs.dense_digraph(n, 31, 0 if kind == "real" else 1, 1 if kind == "real" else 100, kind=kind, device=DEV)
    D = torch.empty_like(W)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    assert apsp.apsp_device_status(clear=True) in (apsp.APSP_OK, apsp.APSP_ETIMEOUT)
    apsp.apsp_fw_ex(W, D, P, bs=64, dtype=apsp.DTYPE_F32, flags=apsp.FLAG_TEST_PANEL_TIMEOUT)
    torch.cuda.synchronize()
    assert apsp.apsp_device_status() == apsp.APSP_ETIMEOUT
    assert apsp.apsp_device_status(clear=True) == apsp.APSP_ETIMEOUT
    assert apsp.apsp_device_status() == apsp.APSP_OK
    # a normal solve on the same context is exact
    apsp.apsp_fw_ex(W, D, P, bs=64, dtype=apsp.DTYPE_F32)
    torch.cuda.synchronize()
    Dr, Pr = oracle.fw_blocked(W.cpu().numpy(), 64)
    np.testing.assert_array_equal(D.cpu().numpy(), Dr)
    np.testing.assert_array_equal(P.cpu().numpy(), Pr)
    assert apsp.apsp_device_status() == apsp.APSP_OK


def test_expired_panel_wait_on_the_16_bit_path():
    n = 256
    W = inputs.dense_digraph(n, 33, 1, 2, device=DEV)  # 16-bit eligible
    D = torch.empty_like(W)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_device_status(clear=True)
    info = apsp.apsp_fw_ex(W, D, P, bs=64, dtype=apsp.DTYPE_U16X2, flags=apsp.FLAG_TEST_PANEL_TIMEOUT)
    torch.cuda.synchronize()
    assert info.dtype_used == apsp.DTYPE_U16X2
    assert apsp.apsp_device_status(clear=True) == apsp.APSP_ETIMEOUT
    apsp.apsp_fw_ex(W, D, P, bs=64, dtype=apsp.DTYPE_U16X2)
    torch.cuda.synchronize()
    Dr, Pr = oracle.fw_blocked(W.cpu().numpy(), 64)
    np.testing.assert_array_equal(D.cpu().numpy(), Dr)
    np.testing.assert_array_equal(P.cpu().numpy(), Pr)
    assert apsp.apsp_device_status() == apsp.APSP_OK


def test_host_entry_point_returns_the_timeout():
    n = 200
    W = inputs.dense_digraph(n, 32, 1, 50)
    D = torch.empty((n, n))
    P = torch.empty((n, n), dtype=torch.int32)
    apsp.apsp_device_status(clear=True)
    with pytest.raises(apsp.ApspError) as e:
        apsp.apsp_fw_host(W, D, P, bs=64, dtype=apsp.DTYPE_F32, flags=apsp.FLAG_TEST_PANEL_TIMEOUT)
    assert e.value.status == apsp.APSP_ETIMEOUT
    assert apsp.apsp_device_status() == apsp.APSP_OK  # the host call cleared it
    apsp.apsp_fw_host(W, D, P, bs=64, dtype=apsp.DTYPE_F32)
    Dr, Pr = oracle.fw_blocked(W.numpy(), 64)
    np.testing.assert_array_equal(D.numpy(), Dr)
    np.testing.assert_array_equal(P.numpy(), Pr)
