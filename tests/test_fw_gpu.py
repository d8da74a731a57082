"""GPU parity of the single-graph path (apsp_fw / apsp_fw_ex / apsp_fw_host)
against the serial oracle.

D and P must match oracle.fw_blocked with the same block size bit for bit:
the kernels perform the same fp32 additions (or exact 16-bit sums) and the
same strict-'<' first-k choice as the serial loop, for integer and real
weights alike. At the full benchmark sizes the oracle cannot run the whole
matrix, so sampled rows are checked against the oracle's Dijkstra (exact for
integer weights, 1e-5 relative for real weights, the tolerance the workload
specification states) and sampled pairs against the oracle's P-walk check.
"""

import numpy as np
import pytest
import torch

import oracle
import paper_1811_01201_gb300 as apsp
from paper_1811_01201_gb300 import inputs
from tests.helpers import all_pairs, load_golden, random_pairs

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")
INF = float("inf")


def _run(W: torch.Tensor, bs=0, dtype=apsp.DTYPE_AUTO, validate=True):
    n = W.shape[0]
    Wd = W.to(DEV)
    D = torch.empty_like(Wd)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    info = apsp.apsp_fw_ex(Wd, D, P, bs=bs, dtype=dtype, validate=validate)
    torch.cuda.synchronize()
    return D.cpu().numpy(), P.cpu().numpy(), info


def _expect_exact(W, D, P, bs):
    Dr, Pr = oracle.fw_blocked(W.numpy() if isinstance(W, torch.Tensor) else W, bs)
    np.testing.assert_array_equal(D, Dr)
    np.testing.assert_array_equal(P, Pr)


# ---------------------------------------------------------------- exact parity, small and ragged n

@pytest.mark.parametrize("n", [1, 2, 5, 31, 32, 33, 127, 128, 129, 200, 256, 300, 384])
@pytest.mark.parametrize("bs", [32, 64, 128])
def test_f32_int_weights_bit_exact(n, bs):
    W = inputs.dense_digraph(n, seed=1000 + n, lo=1, hi=100, density=0.6)
    D, P, info = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
    assert info.bs_used == bs and info.dtype_used == apsp.DTYPE_F32
    _expect_exact(W, D, P, bs)


@pytest.mark.parametrize("n,bs", [(160, 32), (257, 64), (512, 64), (390, 128)])
def test_f32_real_weights_bit_exact(n, bs):
    # real weights take the rescan path for P; the fp32 sums are the same ops
    W = inputs.dense_digraph(n, seed=2000 + n, kind="real", density=0.8)
    D, P, info = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
    _expect_exact(W, D, P, bs)


def test_f32_large_distances_take_generic_path():
    # weights up to 1e6: panel sums exceed the exact-key bound, forcing the rescan path
    W = inputs.dense_digraph(300, seed=7, lo=1, hi=1_000_000, density=0.3)
    D, P, _ = _run(W, bs=64, dtype=apsp.DTYPE_F32)
    _expect_exact(W, D, P, 64)


@pytest.mark.parametrize("bs", [32, 64, 128])
@pytest.mark.parametrize("scale", [1, 2])
def test_f32_keys_near_exactness_bound(bs, scale):
    # integer distances close to the largest panel sum the exact-key path of phase 3 accepts for
    # this BS (keys 2^23 + 2*BS*(a+b) + k + 1 below 2^24: a + b <= 131055, 65519, 32751), and
    # twice that, where rounds fall back to the generic search
    hi = {32: 60000, 64: 30000, 128: 15000}[bs] * scale
    W = inputs.dense_digraph(300, seed=40 + bs, lo=hi // 2, hi=hi, density=0.4)
    D, P, _ = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
    _expect_exact(W, D, P, bs)


@pytest.mark.parametrize("bs", [32, 64, 128])
@pytest.mark.parametrize("n", [256, 300])
def test_f32_complete_graph_with_heavy_old_values(bs, n):
    # light edges around the first 160 vertices make the early rounds keyed while the old values
    # of the other pairs sit at 32767, whose key 2^23 + 256 * 32767 at BS = 128 is the clamp
    # value itself (and at n = 300 the working matrix also holds INF padding)
    W = inputs.dense_digraph(n, seed=70 + bs, lo=1, hi=10)
    heavy = torch.full((n, n), 32767.0)
    hub = torch.zeros(n, dtype=torch.bool)
    hub[:160] = True
    W = torch.where(hub[:, None] | hub[None, :], W, heavy)
    W.fill_diagonal_(0.0)
    D, P, _ = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
    _expect_exact(W, D, P, bs)
    assert int((D == 32767.0).sum()) == 0  # every heavy pair found a path through the hub


def test_config_n512_dense_int():
    # the small benchmark workload: n=512, integer weights in [1,100], dense
    W = inputs.dense_digraph(512, seed=1, lo=1, hi=100)
    for bs in (32, 64):
        D, P, _ = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
        _expect_exact(W, D, P, bs)


@pytest.mark.parametrize("n,hi,bs", [(130, 2, 32), (300, 100, 64), (520, 20, 32), (256, 255, 128), (389, 60, 128)])
def test_u16_path_bit_exact(n, hi, bs):
    W = inputs.dense_digraph(n, seed=3000 + n, lo=1, hi=hi, density=0.5)
    assert hi * (n - 1) < 65535
    D, P, info = _run(W, bs=bs, dtype=apsp.DTYPE_AUTO)
    assert info.dtype_used == apsp.DTYPE_U16X2
    _expect_exact(W, D, P, bs)
    D2, P2, info2 = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
    assert info2.dtype_used == apsp.DTYPE_F32
    np.testing.assert_array_equal(D, D2)
    np.testing.assert_array_equal(P, P2)


def test_u16_bound_edge():
    # max_w*(n-1) = 65534 is eligible; one more unit of weight is not
    n = 257
    W = inputs.dense_digraph(n, seed=5, lo=1, hi=255, density=1.0)
    W[0, 1] = 255.0
    D, P, info = _run(W, bs=32)
    assert info.dtype_used == apsp.DTYPE_U16X2  # 255 * 256 = 65280 < 65535
    _expect_exact(W, D, P, 32)
    W[0, 1] = 300.0  # 300 * 256 = 76800, but the graph is complete: still eligible
    D, P, info = _run(W, bs=32)
    assert info.dtype_used == apsp.DTYPE_U16X2
    _expect_exact(W, D, P, 32)
    W[5, 9] = INF  # one absent edge: the path-length rule alone decides, and 76800 >= 65535
    D, P, info = _run(W, bs=32)
    assert info.dtype_used == apsp.DTYPE_F32
    _expect_exact(W, D, P, 32)
    with pytest.raises(apsp.ApspError) as e:
        _run(W, bs=32, dtype=apsp.DTYPE_U16X2)
    assert e.value.status == apsp.APSP_EINVAL


@pytest.mark.parametrize("n,hi,bs", [(600, 1000, 64), (513, 65534, 32), (1000, 30000, 128)])
def test_u16_path_on_complete_graphs(n, hi, bs):
    # complete graphs: no distance exceeds its direct edge, so integer weights below 65535 are
    # eligible at any n (max_w * (n - 1) is far above 65535 here); D and P equal the fp32 path's
    W = inputs.dense_digraph(n, seed=3500 + n, lo=1, hi=hi)
    D, P, info = _run(W, bs=bs, dtype=apsp.DTYPE_AUTO)
    assert info.dtype_used == apsp.DTYPE_U16X2
    _expect_exact(W, D, P, bs)
    D2, P2, info2 = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
    np.testing.assert_array_equal(D, D2)
    np.testing.assert_array_equal(P, P2)


def test_u16_long_chain_saturation():
    # a directed chain with weight 255 reaches 255*(n-1) = 65280: near the top of the 16-bit range
    n = 257
    W = torch.full((n, n), INF)
    W.fill_diagonal_(0)
    for t in range(n - 1):
        W[t, t + 1] = 255
    W[n - 1, 0] = 1
    D, P, info = _run(W, bs=32)
    assert info.dtype_used == apsp.DTYPE_U16X2
    _expect_exact(W, D, P, 32)


# ---------------------------------------------------------------- special graphs and fixtures

@pytest.mark.parametrize("name", ["tie_break_4.txt", "blocked_vs_naive_4.txt"])
def test_golden_fixtures_on_gpu(name):
    g = load_golden(name)
    # the fixtures use BS=2; with BS >= n the run is one round = naive FW
    D, P, _ = _run(torch.from_numpy(g["W"]), bs=32, dtype=apsp.DTYPE_F32)
    np.testing.assert_array_equal(D, g["D_naive"])
    np.testing.assert_array_equal(P, g["P_naive"])


def test_all_inf_graph_and_single_vertex():
    W = torch.full((150, 150), INF)
    D, P, _ = _run(W, bs=32, dtype=apsp.DTYPE_F32)
    expect = np.full((150, 150), np.inf, np.float32)
    np.fill_diagonal(expect, 0)
    np.testing.assert_array_equal(D, expect)
    assert (P == -1).all()
    D, P, _ = _run(torch.zeros((1, 1)), bs=32)
    assert D[0, 0] == 0 and P[0, 0] == -1


def test_complete_unit_graph_no_improvement():
    n = 200
    W = torch.ones((n, n))
    D, P, _ = _run(W, bs=64, dtype=apsp.DTYPE_F32)
    expect = np.ones((n, n), np.float32)
    np.fill_diagonal(expect, 0)
    np.testing.assert_array_equal(D, expect)
    assert (P == -1).all()


def test_nonzero_input_diagonal_is_ignored():
    W = inputs.dense_digraph(140, seed=9, lo=1, hi=50)
    W.fill_diagonal_(7.0)
    D, P, _ = _run(W, bs=32, dtype=apsp.DTYPE_F32)
    assert (np.diag(D) == 0).all()
    W0 = W.clone()
    W0.fill_diagonal_(0)
    _expect_exact(W0, D, P, 32)


# ---------------------------------------------------------------- API behaviour

def test_in_place_and_workspace():
    n = 256
    W = inputs.dense_digraph(n, seed=11, lo=1, hi=1000, density=0.5)
    Dr, Pr = oracle.fw_blocked(W.numpy(), 64)
    A = W.to(DEV).clone()
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    apsp.apsp_fw_ex(A, A, P, bs=64, dtype=apsp.DTYPE_F32)  # W aliases D
    torch.cuda.synchronize()
    np.testing.assert_array_equal(A.cpu().numpy(), Dr)
    np.testing.assert_array_equal(P.cpu().numpy(), Pr)
    n2 = 200
    W2 = inputs.dense_digraph(n2, seed=12, lo=1, hi=100)
    ws = torch.empty(apsp.apsp_fw_workspace_size(n2, bs=64), dtype=torch.uint8, device=DEV)
    D2 = torch.empty((n2, n2), device=DEV)
    P2 = torch.empty((n2, n2), dtype=torch.int32, device=DEV)
    apsp.apsp_fw_ex(W2.to(DEV), D2, P2, bs=64, workspace=ws)
    torch.cuda.synchronize()
    _expect_exact(W2, D2.cpu().numpy(), P2.cpu().numpy(), 64)


def test_solve_captured_in_a_cuda_graph():
    # validate = 0 with a caller workspace: fully asynchronous, so the whole solve (every
    # round's kernels, launched as programmatic dependents) can be captured and replayed
    n = 384
    W = inputs.dense_digraph(n, seed=14, lo=1, hi=500, density=0.6)
    Wd = W.to(DEV)
    D = torch.empty_like(Wd)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    ws = torch.empty(apsp.apsp_fw_workspace_size(n, bs=64, dtype=apsp.DTYPE_F32), dtype=torch.uint8, device=DEV)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        apsp.apsp_fw_ex(Wd, D, P, bs=64, dtype=apsp.DTYPE_F32, validate=False, workspace=ws, stream=s)
    D.fill_(-1.0)
    P.fill_(7)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    Dr, Pr = oracle.fw_blocked(W.numpy(), 64)
    np.testing.assert_array_equal(D.cpu().numpy(), Dr)
    np.testing.assert_array_equal(P.cpu().numpy(), Pr)


def test_default_entry_point_and_stream():
    n = 333
    W = inputs.dense_digraph(n, seed=13, lo=1, hi=1000, density=0.7)
    s = torch.cuda.Stream()
    Wd = W.to(DEV)
    D = torch.empty_like(Wd)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    with torch.cuda.stream(s):
        apsp.apsp_fw(Wd, D, P, stream=s)
    s.synchronize()
    _expect_exact(W, D.cpu().numpy(), P.cpu().numpy(), apsp.apsp_default_bs(n))


def test_host_entry_point():
    n = 300
    W = inputs.dense_digraph(n, seed=14, lo=1, hi=1000, density=0.5).pin_memory()
    D = torch.empty((n, n)).pin_memory()
    P = torch.empty((n, n), dtype=torch.int32).pin_memory()
    info = apsp.apsp_fw_host(W, D, P, bs=32)
    _expect_exact(W, D.numpy(), P.numpy(), info.bs_used)


def test_invalid_inputs_rejected():
    n = 64
    W = inputs.dense_digraph(n, seed=15, lo=1, hi=10)
    for bad in (-1.0, float("nan")):
        Wb = W.clone()
        Wb[3, 5] = bad
        with pytest.raises(apsp.ApspError) as e:
            _run(Wb)
        assert e.value.status == apsp.APSP_EINVAL
    with pytest.raises(apsp.ApspError) as e:
        _run(W, bs=48)
    assert e.value.status == apsp.APSP_EINVAL
    with pytest.raises(apsp.ApspError) as e:
        _run(W, dtype=apsp.DTYPE_U16X2, validate=False)
    assert e.value.status == apsp.APSP_EINVAL
    # the context stays usable after rejected calls
    D, P, _ = _run(W, bs=32)
    _expect_exact(W, D, P, 32)


def test_deterministic_repeats():
    W = inputs.dense_digraph(384, seed=16, kind="real", density=0.9)
    D1, P1, _ = _run(W, bs=64, dtype=apsp.DTYPE_F32)
    D2, P2, _ = _run(W, bs=64, dtype=apsp.DTYPE_F32)
    assert np.array_equal(D1, D2) and np.array_equal(P1, P2)


# ---------------------------------------------------------------- full benchmark sizes (sampled)

def _sampled_check(n, seed, lo, hi, density, kind, bs, n_src=6, n_pairs=1_000_000, dtype=apsp.DTYPE_AUTO,
                   expect_dtype=None, expect_bs=None):
    Wd = inputs.dense_digraph(n, seed, lo, hi, density=density, kind=kind, device=DEV)
    D = torch.empty_like(Wd)
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    info = apsp.apsp_fw_ex(Wd, D, P, bs=bs, dtype=dtype)
    torch.cuda.synchronize()
    if expect_dtype is not None:
        assert info.dtype_used == expect_dtype
    if expect_bs is not None:
        assert info.bs_used == expect_bs
    W = Wd.cpu().numpy()
    del Wd
    Dh = D.cpu().numpy()
    Ph = P.cpu().numpy()
    del D, P
    torch.cuda.empty_cache()
    rng = np.random.default_rng(seed)
    exact = kind == "int"
    assert (np.diag(Dh) == 0).all()
    for s in rng.choice(n, size=n_src, replace=False):
        ref = oracle.dijkstra(W, int(s))
        row = Dh[s].astype(np.float64)
        if exact:
            np.testing.assert_array_equal(row, ref)
        else:
            fin = np.isfinite(ref)
            assert (np.isfinite(row) == fin).all()
            np.testing.assert_allclose(row[fin], ref[fin], rtol=1e-5)
        assert oracle.check_bellman_row(W, Dh[s], rtol=0.0 if exact else 1e-5) == 0
    pairs = random_pairs(n, n_pairs, seed + 1)
    assert oracle.check_paths(W, Dh, Ph, pairs, rtol=0.0 if exact else 1e-5) == 0


def test_full_n8192_int_density_half():
    _sampled_check(8192, 2, 1, 1000, 0.5, "int", bs=64, expect_dtype=apsp.DTYPE_F32)


@pytest.mark.slow
def test_full_n32768_int():
    _sampled_check(32768, 3, 1, 1000, 1.0, "int", bs=64, n_src=4, dtype=apsp.DTYPE_F32, expect_dtype=apsp.DTYPE_F32)


@pytest.mark.slow
def test_full_n32768_int_auto_takes_the_16_bit_path():
    # the same complete graph with dtype AUTO: no distance exceeds its direct edge (<= 1000), so the
    # exact 16-bit path runs
    _sampled_check(32768, 3, 1, 1000, 1.0, "int", bs=0, n_src=4, expect_dtype=apsp.DTYPE_U16X2)


@pytest.mark.slow
def test_full_n32768_real():
    _sampled_check(32768, 4, 0, 1, 1.0, "real", bs=64, n_src=4, dtype=apsp.DTYPE_F32)


@pytest.mark.slow
def test_full_n32768_u16():
    _sampled_check(32768, 5, 1, 2, 1.0, "int", bs=64, n_src=4, expect_dtype=apsp.DTYPE_U16X2)


@pytest.mark.slow
def test_full_n32768_u16_default_block_size():
    # the benchmark's 16-bit run: library default block size (128 on this path above n = 16384)
    _sampled_check(32768, 5, 1, 2, 1.0, "int", bs=0, n_src=4, expect_dtype=apsp.DTYPE_U16X2, expect_bs=128)


def _host_available_bytes() -> int:
    with open("/proc/meminfo") as f:
        for line in f:
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    return 0


@pytest.mark.slow
def test_max_n65536_int_in_place():
    # The largest n the library accepts: element offsets pass 2^31 and 2^32. Solved in place
    # (W aliases D) to keep the device at 32 GiB; the host keeps W only (16 GiB). Sampled rows
    # of D against Dijkstra, the optimality condition on those rows, and every P entry of
    # those rows: -1 only where D is the direct edge, else an intermediate k with
    # D[s][j] == D[s][k] + D[k][j] (exact for integer weights).
    n, seed = 65536, 6
    if _host_available_bytes() < (n * n * 4) + (32 << 30):
        pytest.skip("not enough free host memory for a 16 GiB copy of W")
    if torch.cuda.mem_get_info()[0] < 2 * n * n * 4 + (8 << 30):
        pytest.skip("not enough free device memory for D and P at n=65536")
    D = inputs.dense_digraph(n, seed, 1, 1000, device=DEV)
    W = D.cpu().numpy()
    P = torch.empty((n, n), dtype=torch.int32, device=DEV)
    info = apsp.apsp_fw_ex(D, D, P, dtype=apsp.DTYPE_F32)
    torch.cuda.synchronize()
    assert info.dtype_used == apsp.DTYPE_F32 and info.bs_used == 64
    rng = np.random.default_rng(seed)
    cols = torch.arange(n, device=DEV)
    for s in [0, n - 1] + [int(v) for v in rng.choice(n, size=2, replace=False)]:
        row = D[s].cpu().numpy()
        np.testing.assert_array_equal(row.astype(np.float64), oracle.dijkstra(W, s))
        assert oracle.check_bellman_row(W, row) == 0
        k = P[s].long()
        direct = k < 0
        via = D[k.clamp(min=0), cols].cpu().numpy()
        kh, dh = k.cpu().numpy(), direct.cpu().numpy()
        w = W[s].copy()
        w[s] = 0.0
        np.testing.assert_array_equal(row[dh], w[dh])
        j = np.nonzero(~dh)[0]
        assert ((kh[j] != s) & (kh[j] != j) & (kh[j] < n)).all()
        np.testing.assert_array_equal(row[j], row[kh[j]] + via[j])
    del D, P
    torch.cuda.empty_cache()


def test_autotuner_returns_a_valid_block_size():
    bs, ms = apsp.apsp_autotune_bs(1024)
    assert bs in (32, 64, 128)
    assert all(t > 0 for t in ms)
    assert ms[(32, 64, 128).index(bs)] == min(ms)
    W = inputs.dense_digraph(1024, seed=77, lo=1, hi=100, density=0.5)
    D, P, info = _run(W, bs=bs, dtype=apsp.DTYPE_F32)
    assert info.bs_used == bs
    _expect_exact(W, D, P, bs)
