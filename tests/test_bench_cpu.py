"""CPU checks of bench.py's host logic: the reference arm (the serial oracle),
its JSON line, and the multi-process path (world size 2 over gloo)."""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_reference_arm_single_process():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                          "--ref-sample-n", "96"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GFLOPS" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_two_ranks_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-sample-n", "64"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    assert json.loads(lines[0])["n_gpus"] == 2


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    v = bench.max_over_ranks(10.0 + rank * 5.0, world, torch.device("cpu"))
    q.put((rank, v))
    dist.destroy_process_group()


def test_max_over_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert got == {0: 15.0, 1: 15.0}


def test_profile_traffic_parser(tmp_path, monkeypatch):
    # the summary's value may carry a note after the number; the kernel-source hash gates it
    sys.path.insert(0, ROOT)
    import hashlib

    import bench
    src = tmp_path / "kernel.cuh"
    src.write_text("// kernel\n")
    h = hashlib.sha256(src.read_bytes()).hexdigest()[:16]
    summ = tmp_path / "summary.md"
    summ.write_text(f"# x\n\n- kernel_source_sha256_16: `{h}`\n- dram_bytes_per_launch: 100.0e6   (mean)\n")
    monkeypatch.setattr(bench, "KERNEL_SRC", str(src))
    monkeypatch.setattr(bench, "PROFILE_SUMMARY", {"int": str(summ), "real": str(summ)})
    scale = ((32768 - 64) / (bench.PROFILE_N - bench.PROFILE_BS)) ** 2
    assert bench._traffic_from_profile(32768, 64) == pytest.approx(100.0e6 * scale)
    assert bench._traffic_from_profile(32768, 128) is None          # other block size
    src.write_text("// changed kernel\n")
    assert bench._traffic_from_profile(32768, 64, "real") is None   # stale capture


def test_clock_sampler_summary_reasons():
    # rows as nvidia-smi prints them (noheader, nounits): index, sm MHz, max MHz, power,
    # active mask, hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.rows = [["0", "2070", "2070", "900.1", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["0", "1950", "2070", "1400.0", "0x4", "Not Active", "Not Active", "Not Active", "Active"],
               ["0", "2070", "2070", "1200.0", "0x0", "Not Active", "Not Active", "Not Active", "Not Active"],
               ["0", "[N/A]", "2070"]]  # a malformed sample is skipped
    sm = cs.summary()
    assert sm["sm_mhz"] == 2070.0 and sm["sm_max_mhz"] == 2070.0 and sm["samples"] == 3
    assert sm["reasons"] == ["sw_power_cap"]
    cs.rows.append(["0", "1200", "2070", "600.0", "0x40", "Not Active", "Active", "Not Active", "Not Active"])
    assert "hw_thermal_slowdown" in cs.summary()["reasons"]
