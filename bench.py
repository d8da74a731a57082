"""Benchmark: blocked Floyd-Warshall APSP on one GB300 (and N independent replicas).

Default workload (one "step" = one full all-pairs shortest-paths solve, all
three phases of every block round, through the library's C ABI):
  dense random digraph, n = 32768, fp32 integer weights uniform in [1, 1000],
  zero diagonal, int32 path matrix -- 4 GiB D + 4 GiB P, far larger than L2,
  so no cache flush is needed between steps.
Metric: APSP GFLOPS = 2 n^3 / step time (the 2n^3 convention: one add and one
compare per relaxation, n^3 relaxations).

Printed JSON line (rank 0): value (device-timed, inputs resident in HBM),
e2e (same metric through apsp_fw_host with host buffers, copies included),
roofline of the dominant kernel (phase 3, bound by the ALU pipe that
executes FMNMX), cpu_baseline (the serial oracle on a bounded sample), clocks
sampled during the timed region, and the 16-bit path on the n = 32768,
weights in [1, 2] workload as an extra key.

`--impl reference` times the serial C oracle instead (this repository has no
other reference implementation), on a bounded sample per step.

Multi-GPU: every graph is independent, so N ranks run N independent replicas
("replicas only", weak scaling; no collective on the data path).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Roofline denominators (unit counts x clock). Issue rates measured with a
# register-operand microbenchmark on a GB300 (relaxations per SM clock): 152
# SMs, one warp instruction per clock per SM sub-partition (128 lanes/clk/SM).
# The FP32 min issues at full rate, and the three-input min the compiler forms
# from two successive mins at half rate, so one relaxation costs one min lane:
# 128 relaxations/clk/SM. The fp32 pattern (add.rn.f32x2 + two mins per k pair)
# also takes two issue slots per two relaxations, the same bound. The 16-bit
# pattern (add.u16x2 + min.u16x2, two relaxations each) is issue-bound at the
# same 128. Peak "flops"/s = 2 * 152 * 128 * f in the 2n^3 convention.
SMS = 152
SM_MAX_MHZ = 2070.0
ALU_PEAK_F32_TFLOPS = 2 * SMS * 128 * SM_MAX_MHZ * 1e6 / 1e12     # 80.54
ALU_PEAK_U16_TFLOPS = 2 * SMS * 128 * SM_MAX_MHZ * 1e6 / 1e12     # 80.54
# What the fp32 phase-3 hot loop reaches with its panel pairs in shared memory and
# no global traffic (8x8 register tile, 2 CTAs/SM; relaxations per SM clock from
# ncu cycle counts): the instruction mix is bound by operand reads from the
# register file, not by the min or add pipes (issue active 56%).
HOT_LOOP_CEILING_F32_TFLOPS = 2 * SMS * 65.5 * SM_MAX_MHZ * 1e6 / 1e12  # 41.2


def _hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s (no measured peak file)"


HBM_PEAK_GBS, HBM_PEAK_SOURCE = _hbm_peak()

PROFILE_SUMMARY = {"int": os.path.join(ROOT, "profiles", "phase3_f32_n8192_bs64.md"),
                   "real": os.path.join(ROOT, "profiles", "phase3_f32_real_n8192_bs64.md")}
PROFILE_N, PROFILE_BS = 8192, 64  # workload of that capture
KERNEL_SRC = os.path.join(ROOT, "paper_1811_01201_gb300", "csrc", "fw_minplus_f32.cuh")


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows: list[list[str]] = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=5)
                for line in out.stdout.strip().splitlines():
                    self.rows.append([x.strip() for x in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        if self._t:
            self._t.join(timeout=10)

    def summary(self) -> dict:
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def _traffic_from_profile(n: int, bs: int, kind: str = "int"):
    """Per-launch DRAM bytes of the phase-3 kernel from the committed ncu summary of the weight
    kind (captured at n=8192), scaled to this n by the tile count ((n-BS)^2), or None when the
    summary is missing, the block size differs, or the kernel source changed since the capture."""
    if bs != PROFILE_BS:
        return None
    try:
        text = open(PROFILE_SUMMARY[kind]).read()
        src_hash = hashlib.sha256(open(KERNEL_SRC, "rb").read()).hexdigest()[:16]
    except OSError:
        return None
    got = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            got[k.strip()] = v.strip().strip("`")
    if got.get("kernel_source_sha256_16") != src_hash:
        return None
    try:
        return float(got["dram_bytes_per_launch"].split()[0]) * ((n - bs) / (PROFILE_N - PROFILE_BS)) ** 2
    except (KeyError, ValueError):
        return None


def max_over_ranks(x: float, world: int, device) -> float:
    """Largest value of x over all ranks (the slowest replica sets the job time)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle legs

def _oracle_sample(n_full: int, seed: int, lo: int, hi: int, n_sample: int, bs: int, kind: str = "int"):
    import oracle
    from paper_1811_01201_gb300 import inputs
    W = inputs.dense_digraph(n_full, seed, lo, hi, kind=kind, rows=(0, n_sample))[:, :n_sample].contiguous().numpy()
    t0 = time.perf_counter()
    oracle.fw_blocked(W, bs)
    dt = time.perf_counter() - t0
    return dt, 2.0 * n_sample ** 3


def cpu_baseline(args) -> dict:
    """The serial oracle's naive Floyd-Warshall (Section 3) on one host core: the whole n=512
    workload, and a rate sample on the leading block of the timed workload; the full-size
    times are extrapolated from the sample as t * (n / sample)^3 and labelled so."""
    import oracle
    from paper_1811_01201_gb300 import inputs
    m = args.cpu_sample_n
    W = inputs.dense_digraph(args.n, args.seed, 1, 1000, kind=args.kind, rows=(0, m))[:, :m].contiguous().numpy()
    t0 = time.perf_counter()
    oracle.fw_naive(W)
    dt = time.perf_counter() - t0
    W5 = inputs.dense_digraph(512, 1, 1, 100).numpy()
    t1 = time.perf_counter()
    oracle.fw_naive(W5)
    dt5 = time.perf_counter() - t1
    rate = 2.0 * m ** 3 / dt
    return {"value": round(rate / 1e9, 4), "unit": "GFLOPS", "cores": 1, "kind": "oracle",
            "sample": f"serial C naive FW (oracle_fw_naive) on a sample: the leading {m}x{m} block of the "
                      f"n={args.n} workload, {dt:.1f} s; rate of that sample",
            "n512_s": round(dt5, 4), "n512_gflops": round(2.0 * 512 ** 3 / dt5 / 1e9, 4),
            "n8192_s_extrapolated": round(dt * (8192 / m) ** 3, 1),
            f"n{args.n}_s_extrapolated": round(dt * (args.n / m) ** 3, 1)}


def cpu_parallel_baseline(args) -> dict:
    """The paper's blocked design on all host cores (OpenMP; oracle/host_blocked.c, bit-exact
    with the serial oracle), timed on the leading block of the same workload."""
    from oracle import host_blocked
    from paper_1811_01201_gb300 import inputs
    m = args.cpu_par_sample_n
    W = inputs.dense_digraph(args.n, args.seed, 1, 1000, kind=args.kind, rows=(0, m))[:, :m].contiguous().numpy()
    host_blocked.build()
    t0 = time.perf_counter()
    host_blocked.fw_blocked(W, args.bs)
    dt = time.perf_counter() - t0
    return {"value": round(2.0 * m ** 3 / dt / 1e9, 3), "unit": "GFLOPS", "cores": host_blocked.threads(),
            "kind": "the paper's blocked design on the host cores (OpenMP over blocks, vectorised j loop)",
            "sample": f"blocked FW (BS={args.bs}) on the leading {m}x{m} block of the n={args.n} workload, "
                      f"{dt:.1f} s"}


def run_reference(args, rank: int, world: int):
    if rank != 0:
        return
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        _oracle_sample(args.n, args.seed, 1, 1000, args.ref_sample_n, args.bs, args.kind)
    times = []
    flops = 0.0
    for _ in range(args.steps):
        dt, fl = _oracle_sample(args.n, args.seed, 1, 1000, args.ref_sample_n, args.bs, args.kind)
        times.append(dt)
        flops = fl
    tot = sum(times)
    val = flops * args.steps / tot / 1e9
    line = {"impl": "reference", "metric": "APSP GFLOPS (2n^3/s)", "value": round(val, 4), "unit": "GFLOPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(tot / args.steps * 1e3, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": _config(args),
            "cpu_baseline": {"value": round(val, 4), "unit": "GFLOPS", "cores": 1, "kind": "oracle",
                             "sample": f"serial C blocked FW (BS={args.bs}) on the leading "
                                       f"{args.ref_sample_n}x{args.ref_sample_n} block of the n={args.n} workload "
                                       "per step"},
            "e2e": {"value": round(val, 4), "unit": "GFLOPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _config(args) -> dict:
    wdesc = "fp32 integer weights U[1,1000]" if args.kind == "int" else "fp32 real weights U(0,1]"
    return {"workload": f"dense random digraph n={args.n}, {wdesc}, zero diagonal, "
                        "int32 path matrix (blocked Floyd-Warshall, one full solve per step)",
            "n": args.n, "bs": args.bs, "weights": "int [1,1000]" if args.kind == "int" else "real (0,1]",
            "density": 1.0,
            "l2": "inputs larger than L2 (4 GiB D + 4 GiB P at n=32768); no flush"}


# ---------------------------------------------------------------- GPU leg

def run_gpu(args, rank: int, world: int):
    import torch
    import torch.distributed as dist

    import paper_1811_01201_gb300 as apsp
    from paper_1811_01201_gb300 import inputs

    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    apsp.load(build_if_missing=True)
    n = args.n
    s = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    W = inputs.dense_digraph(n, args.seed, 1, 1000, kind=args.kind, device=dev)
    D = torch.empty_like(W)
    P = torch.empty((n, n), dtype=torch.int32, device=dev)
    ws = torch.empty(apsp.apsp_fw_workspace_size(n, bs=args.bs, dtype=apsp.DTYPE_F32), dtype=torch.uint8,
                     device=dev)

    def step(flags=0):
        return apsp.apsp_fw_ex(W, D, P, bs=args.bs, dtype=apsp.DTYPE_F32, validate=True, workspace=ws,
                               flags=flags)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # Timed region: K steps bracketed by barrier + synchronize; phase-3 launches
    # timed with CUDA events on the launching stream inside the library.
    ph_ms = [0.0, 0.0, 0.0]
    ph_launch = [0, 0, 0]
    launches = 0
    info = None
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        marks = []
        for _ in range(args.steps):
            info = step()
            launches += info.launches
            marks.append(torch.cuda.Event(enable_timing=True))
            marks[-1].record(s)
        e1.record(s)
        torch.cuda.synchronize()
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), world, dev)
    per_step = [e0.elapsed_time(marks[0])] + [marks[i - 1].elapsed_time(marks[i]) for i in range(1, len(marks))]
    # Per-phase device time from separate steps that record an event after every launch (the
    # events keep each launch from overlapping its predecessor, so these steps run apart from
    # the timed ones).
    ph_steps = min(args.steps, 3)
    for _ in range(ph_steps):
        info = step(flags=apsp.FLAG_TIME_PHASES)
        for q in range(3):
            ph_ms[q] += info.phase_ms[q]
            ph_launch[q] += info.phase_launches[q]
    flops = 2.0 * n ** 3
    value = flops * args.steps * world / (ms * 1e-3) / 1e9

    # Phase-3 roofline: algorithmic relaxations of all phase-3 launches
    # ((n - BS)^2 * BS per round, 2 flops each) / their summed event time.
    R = n // args.bs
    ph3_flops = 2.0 * (n - args.bs) ** 2 * args.bs * (R) * ph_steps
    ph3_tflops = ph3_flops / (ph_ms[2] * 1e-3) / 1e12 if ph_ms[2] > 0 else None
    roof = {"bound": "alu", "achieved": round(ph3_tflops, 3) if ph3_tflops else None,
            "peak": round(ALU_PEAK_F32_TFLOPS, 2), "unit": "TFLOP/s",
            "frac": round(ph3_tflops / ALU_PEAK_F32_TFLOPS, 4) if ph3_tflops else None,
            "traffic": _traffic_from_profile(n, args.bs, args.kind),
            "kernel": f"fw_phase3_f32_real_kernel<{args.bs}>" if args.kind == "real" else f"fw_phase3_f32_kernel<{args.bs}>",
            "peak_source": "derived: 152 SMs x 128 relaxations/clk (one min lane each; FP32 min and "
                           "three-input min issue rates measured on a GB300) x 2070 MHz x 2 flop",
            "hot_loop_ceiling_tflops": round(HOT_LOOP_CEILING_F32_TFLOPS, 2),
            "frac_of_hot_loop_ceiling": round(ph3_tflops / HOT_LOOP_CEILING_F32_TFLOPS, 4) if ph3_tflops else None,
            "phase_ms_per_step": [round(x / ph_steps, 3) for x in ph_ms],
            "phase_launches_per_step": [x // ph_steps for x in ph_launch],
            "phase_steps": ph_steps}
    # Phases 1 and 2 are latency-bound sequential sweeps: their HBM rate against the copy peak.
    # Algorithmic bytes per tile: BS^2 * (4 read + 4 D write + 4 P write).
    tile_b = 12.0 * args.bs * args.bs
    ph12 = {"phase1_us_per_launch": round(ph_ms[0] * 1e3 / max(1, ph_launch[0]), 2),
            "phase2_us_per_launch": round(ph_ms[1] * 1e3 / max(1, ph_launch[1]), 2),
            "algorithmic_bytes_per_launch": [tile_b, tile_b * 2 * (R - 1)]}
    if ph_ms[0] > 0 and ph_ms[1] > 0:
        g1 = tile_b * ph_launch[0] / (ph_ms[0] * 1e-3) / 1e9
        g2 = tile_b * 2 * (R - 1) * ph_launch[1] / (ph_ms[1] * 1e-3) / 1e9
        ph12 |= {"achieved_gbs": [round(g1, 2), round(g2, 1)], "peak_gbs": HBM_PEAK_GBS,
                 "frac": [round(g1 / HBM_PEAK_GBS, 5), round(g2 / HBM_PEAK_GBS, 4)],
                 "peak_source": HBM_PEAK_SOURCE}
    roof["phases_1_2"] = ph12
    clocks = clk.summary()

    line = {"metric": "APSP GFLOPS (2n^3/s)", "value": round(value, 2), "unit": "GFLOPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 3),
            "ms_per_step_min_median_max": [round(min(per_step), 3), round(statistics.median(per_step), 3),
                                           round(max(per_step), 3)],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": _config(args) | {"parallelism": f"replicas x{world}"},
            "gpu_launches": launches, "roofline": roof, "clocks": clocks}

    # Path reconstruction on the device from the solve's P (before anything overwrites it) (apsp_paths), seeded random pairs.
    if args.paths > 0:
        line["paths"] = run_paths(args, dev, P, n, args.paths)

    # End to end through apsp_fw_host: host pinned W in, host D and P out, every step. Timed right
    # after the main solve and its path walk: in one process, after other large solves and their
    # device allocations, the same host copies ran up to 5x slower while every kernel kept its
    # time, so the side workloads come after this measurement.
    if args.e2e:
        Wh = W.cpu().pin_memory()
        Dh = torch.empty((n, n), dtype=torch.float32).pin_memory()
        Ph = torch.empty((n, n), dtype=torch.int32).pin_memory()
        del W, P, ws
        # Copy rates between these pinned buffers and the device, outside the timed region
        # (diagnostic: the e2e time minus the device solve should be about the copies).
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record(s)
        D.copy_(Wh, non_blocking=True)
        c1.record(s)
        Dh.copy_(D, non_blocking=True)
        c2.record(s)
        torch.cuda.synchronize()
        copy_gbs = [round(4 * n * n / (c0.elapsed_time(c1) * 1e-3) / 1e9, 1),
                    round(4 * n * n / (c1.elapsed_time(c2) * 1e-3) / 1e9, 1)]
        del D
        torch.cuda.empty_cache()
        apsp.apsp_fw_host(Wh, Dh, Ph, bs=args.bs, dtype=apsp.DTYPE_F32)
        torch.cuda.synchronize()
        with ClockSampler(local) as eclk:
            barrier()
            t0 = time.perf_counter()
            for _ in range(args.e2e_steps):
                apsp.apsp_fw_host(Wh, Dh, Ph, bs=args.bs, dtype=apsp.DTYPE_F32)
            torch.cuda.synchronize()
            barrier()
            et = (time.perf_counter() - t0) / args.e2e_steps
        line["e2e"] = {"value": round(flops * world / et / 1e9, 2), "unit": "GFLOPS",
                       "h2d_bytes_per_step": 4 * n * n, "d2h_bytes_per_step": 8 * n * n,
                       "ms_per_step": round(et * 1e3, 3), "steps": args.e2e_steps,
                       "api": "apsp_fw_host (pinned host buffers)",
                       "copy_gbs_h2d_d2h": copy_gbs, "clocks": eclk.summary()}
        # the later workloads write their results into D and P
        D = torch.empty((n, n), dtype=torch.float32, device=dev)
        P = torch.empty((n, n), dtype=torch.int32, device=dev)

    # 16-bit exact path on its workload (n, weights in [1,2]: max_w*(n-1) < 65535).
    if args.u16:
        # block size: the library's default for the 16-bit path (128 above n = 16384)
        Wu = inputs.dense_digraph(n, args.seed + 2, 1, 2, device=dev)
        wsu = torch.empty(apsp.apsp_fw_workspace_size(n), dtype=torch.uint8, device=dev)
        for _ in range(max(1, args.warmup - 1)):
            apsp.apsp_fw_ex(Wu, D, P, workspace=wsu)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(s)
        for _ in range(args.steps):
            iu = apsp.apsp_fw_ex(Wu, D, P, workspace=wsu)
        a1.record(s)
        torch.cuda.synchronize()
        ums = a0.elapsed_time(a1) / args.steps
        ip = apsp.apsp_fw_ex(Wu, D, P, workspace=wsu, flags=apsp.FLAG_TIME_PHASES)
        bsu = ip.bs_used
        ph3u = 2.0 * (n - bsu) ** 2 * bsu * (n // bsu) / (ip.phase_ms[2] * 1e-3) / 1e12
        line["u16x2"] = {"workload": f"dense digraph n={n}, integer weights U[1,2] (16-bit eligible)",
                         "value": round(flops / (ums * 1e-3) / 1e9, 2), "unit": "GFLOPS",
                         "ms_per_step": round(ums, 3), "dtype_used": "u16x2" if iu.dtype_used == 2 else "f32",
                         "bs_used": bsu,
                         "phase_ms": [round(x, 3) for x in ip.phase_ms],
                         "phase3_tflops": round(ph3u, 3), "peak_tflops": round(ALU_PEAK_U16_TFLOPS, 2),
                         "phase3_frac": round(ph3u / ALU_PEAK_U16_TFLOPS, 4)}
        del Wu, wsu

    # The other single-graph workloads: n = 512 (integer weights U[1,100], dense), n = 32768 with
    # real weights U(0,1], and a 16-bit-eligible graph whose elements improve (n = 16384,
    # U[1,3], density 0.5: 3 * 16383 < 65535).
    if args.extra_solves:
        line["n512"] = run_solve_key(args, dev, 512, 1, 1, 100, 1.0, "int", 0, apsp.DTYPE_F32,
                                     "dense digraph n=512, integer weights U[1,100]")
        if n == 32768:
            line["real32768"] = run_solve_key(args, dev, n, 4, 0, 1, 1.0, "real", 64, apsp.DTYPE_F32,
                                              "dense digraph n=32768, real weights U(0,1]", D, P, traffic_kind="real")
        line["u16x2_improving"] = run_solve_key(args, dev, 16384, 9, 1, 3, 0.5, "int", 0, apsp.DTYPE_AUTO,
                                                "digraph n=16384, integer weights U[1,3], edge density 0.5 "
                                                "(16-bit eligible; elements improve)", D, P)

    if args.autotune_c2:
        line["n8192_autotuned"] = run_c2(args, dev)
    if args.batched:
        line["batched"] = run_batched(args, dev)
    if args.serve_seconds > 0:
        line["served"] = run_serve(args, dev, args.serve_seconds)

    if rank == 0 and args.cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
        line["cpu_parallel_baseline"] = cpu_parallel_baseline(args)
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_solve_key(args, dev, n, seed, lo, hi, density, kind, bs, dtype, workload, D=None, P=None,
                  traffic_kind=None) -> dict:
    """One more single-graph workload timed like the main one (device events around whole
    solves, warm-ups first), with its phase times from one separate instrumented solve and the
    phase-3 rate against the same ALU peak."""
    import torch

    import paper_1811_01201_gb300 as apsp
    from paper_1811_01201_gb300 import inputs
    W = inputs.dense_digraph(n, seed, lo, hi, density=density, kind=kind, device=dev)
    if D is None or D.numel() != n * n:
        D = torch.empty_like(W)
        P = torch.empty((n, n), dtype=torch.int32, device=dev)
    D, P = D.view(n, n), P.view(n, n)
    ws = torch.empty(apsp.apsp_fw_workspace_size(n, bs=bs, dtype=dtype), dtype=torch.uint8, device=dev)
    s = torch.cuda.current_stream()
    for _ in range(2):
        apsp.apsp_fw_ex(W, D, P, bs=bs, dtype=dtype, workspace=ws)
    torch.cuda.synchronize()
    steps = max(3, min(args.steps, 10))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        info = apsp.apsp_fw_ex(W, D, P, bs=bs, dtype=dtype, workspace=ws)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    ip = apsp.apsp_fw_ex(W, D, P, bs=bs, dtype=dtype, workspace=ws, flags=apsp.FLAG_TIME_PHASES)
    bsu = ip.bs_used
    n_pad = ip.n_pad
    ph3 = 2.0 * (n_pad - bsu) ** 2 * bsu * (n_pad // bsu) / (ip.phase_ms[2] * 1e-3) / 1e12 if ip.phase_ms[2] > 0 else 0
    improved = int((P >= 0).sum())
    out = {"workload": workload, "value": round(2.0 * n ** 3 / (ms * 1e-3) / 1e9, 2), "unit": "GFLOPS",
           "ms_per_step": round(ms, 3), "steps": steps, "bs_used": bsu,
           "dtype_used": "u16x2" if info.dtype_used == apsp.DTYPE_U16X2 else "f32",
           "phase_ms": [round(x, 3) for x in ip.phase_ms], "phase3_tflops": round(ph3, 3),
           "peak_tflops": round(ALU_PEAK_F32_TFLOPS, 2), "phase3_frac": round(ph3 / ALU_PEAK_F32_TFLOPS, 4),
           "p_entries_set": improved, "gpu_launches_per_step": info.launches}
    if traffic_kind is not None:
        out["phase3_traffic_bytes_per_launch"] = _traffic_from_profile(n, bsu, traffic_kind)
    del W, ws
    return out


def run_paths(args, dev, P, n: int, count: int, cap: int = 64, reps: int = 5) -> dict:
    """apsp_paths over `count` seeded random (i, j) pairs of the solved n-vertex graph: one thread
    walks one pair; a path of L vertices costs 2L - 3 dependent random reads of P."""
    import torch

    import paper_1811_01201_gb300 as apsp
    from paper_1811_01201_gb300 import inputs
    pairs = inputs.vertex_pairs(count, n, 11, device=dev)
    out = torch.empty((count, cap), dtype=torch.int32, device=dev)
    lens = torch.empty((count,), dtype=torch.int32, device=dev)
    s = torch.cuda.current_stream()
    for _ in range(3):
        apsp.apsp_paths(P, pairs, cap, out, lens)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(reps):
        apsp.apsp_paths(P, pairs, cap, out, lens)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    L = lens.to(torch.int64)
    ok = L >= 2
    reads = int((2 * L[ok] - 3).sum())
    return {"workload": f"{count} seeded random (i, j) pairs of the timed solve's graph (n={n}), cap {cap}",
            "paths_per_s": round(count / (ms * 1e-3), 1), "ms": round(ms, 4),
            "mean_vertices": round(float(L[ok].float().mean()), 3), "failed": int((L < 0).sum()),
            "same_vertex_pairs": int((L == 1).sum()),
            "p_reads_per_s": round(reads / (ms * 1e-3), 1),
            "sector_gbs": round(32.0 * reads / (ms * 1e-3) / 1e9, 1), "launches_per_call": 1}


def run_extra(args, rank: int, world: int):
    """--workload batched | serve: one JSON line for that workload alone."""
    import torch

    import paper_1811_01201_gb300 as apsp
    local = _env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    apsp.load(build_if_missing=True)
    with ClockSampler(local) as clk:
        if args.workload == "batched":
            r = run_batched(args, dev)
            sizes = f"n={args.batch_n}" if args.batch_n > 0 else "n log-uniform in [16,512]"
            line = {"metric": f"APSP graphs/s ({args.batch_count} graphs, {sizes})", "value": r["graphs_per_s"],
                    "unit": "graphs/s", "gflops": r["gflops"]}
        else:
            r = run_serve(args, dev, args.serve_seconds if args.serve_seconds > 0 else 60.0,
                          sweep_fracs=(0.5, 0.95, 1.1) if args.serve_sweep else None)
            line = {"metric": "APSP served graphs/s at 80% of saturation", "value": r["graphs_per_s"],
                    "unit": "graphs/s", "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"]}
    line.update({"n_gpus": world, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                 "data": "synthetic", "config": {"workload": r["workload"]}, "detail": r, "clocks": clk.summary()})
    if rank == 0:
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- batched and served workloads

def run_c2(args, dev, n=8192, seed=2) -> dict:
    """n=8192, integer weights U[1,1000], edge density 0.5; BS chosen by the library's autotuner."""
    import torch

    import paper_1811_01201_gb300 as apsp
    from paper_1811_01201_gb300 import inputs
    bs, tune_ms = apsp.apsp_autotune_bs(n)
    W = inputs.dense_digraph(n, seed, 1, 1000, density=0.5, device=dev)
    D = torch.empty_like(W)
    P = torch.empty((n, n), dtype=torch.int32, device=dev)
    ws = torch.empty(apsp.apsp_fw_workspace_size(n, bs=bs, dtype=apsp.DTYPE_F32), dtype=torch.uint8, device=dev)
    for _ in range(3):
        apsp.apsp_fw_ex(W, D, P, bs=bs, dtype=apsp.DTYPE_F32, workspace=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(3, args.steps)
    e0.record()
    for _ in range(steps):
        apsp.apsp_fw_ex(W, D, P, bs=bs, dtype=apsp.DTYPE_F32, workspace=ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    return {"workload": "dense random digraph n=8192, integer weights U[1,1000], edge density 0.5",
            "bs_autotuned": bs, "autotune_ms_bs32_64_128": [round(x, 3) for x in tune_ms],
            "value": round(2.0 * n ** 3 / (ms * 1e-3) / 1e9, 1), "unit": "GFLOPS", "ms_per_step": round(ms, 3)}


def run_batched(args, dev, seed=6) -> dict:
    """4096 independent dense digraphs, n log-uniform in [16, 512], integer weights U[1,100],
    density 0.7: one CUDA-graph-captured persistent launch vs one library call per graph.
    --batch-n N gives every graph order N (--batch-count graphs), to study one size alone."""
    import torch

    import paper_1811_01201_gb300 as apsp
    from paper_1811_01201_gb300 import inputs
    count = args.batch_count
    ns = [args.batch_n] * count if args.batch_n > 0 else inputs.batch_sizes(count, seed)
    Ws = [inputs.dense_digraph(n, inputs.batch_graph_seed(seed, g), 1, 100, density=0.7, device=dev)
          for g, n in enumerate(ns)]
    Ds = [torch.empty_like(w) for w in Ws]
    Ps = [torch.empty(w.shape, dtype=torch.int32, device=dev) for w in Ws]
    flops = sum(2.0 * n ** 3 for n in ns)
    s = torch.cuda.Stream(device=dev)
    b = apsp.Batch(Ws, Ds, Ps, stream=s)
    reps = max(3, args.steps)

    def time_graph_replays():
        with torch.cuda.stream(s):
            for _ in range(2):
                b.launch(stream=s)
        s.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            b.launch(stream=s)
        for _ in range(2):
            graph.replay()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps * 1e-3

    t_default = time_graph_replays()   # phase-3 tiles by the size rule
    rows = b.autotune(stream=s)        # phase-3 tiles timed per size class
    t_b = time_graph_replays()
    # one library call per graph (async, no validation): the per-graph launch path
    with torch.cuda.stream(s):
        for g in range(count):
            apsp.apsp_fw_ex(Ws[g], Ds[g], Ps[g], bs=32, dtype=apsp.DTYPE_F32, validate=False, stream=s)
    s.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(s):
        for g in range(count):
            apsp.apsp_fw_ex(Ws[g], Ds[g], Ps[g], bs=32, dtype=apsp.DTYPE_F32, validate=False, stream=s)
    s.synchronize()
    t_s = time.perf_counter() - t0
    b.close()
    sizes = f"n={args.batch_n}" if args.batch_n > 0 else "n log-uniform [16,512]"
    return {"workload": f"{count} dense digraphs, {sizes}, integer weights U[1,100], density 0.7",
            "ph3_tile_rows_by_class": dict(zip(["n<=64", "n<=128", "n<=256", "n<=512"], rows)),
            "graphs_per_s_size_rule_tiles": round(count / t_default, 1),
            "graphs_per_s": round(count / t_b, 1), "gflops": round(flops / t_b / 1e9, 1),
            "ms_per_batch": round(t_b * 1e3, 3), "launch": "one persistent kernel replayed from a CUDA graph",
            "per_graph_calls": {"graphs_per_s": round(count / t_s, 1), "gflops": round(flops / t_s / 1e9, 1),
                                "ms": round(t_s * 1e3, 1)},
            "speedup_vs_per_graph": round(t_s / t_b, 2)}


def run_serve(args, dev, seconds: float, seed=7, pool_size=512, clients=4, sweep_fracs=None,
              sweep_seconds=15.0) -> dict:
    """Poisson stream of requests, n = clip(round(lognormal(ln 256, 1.0)), 32, 4096), integer
    weights U[1,64]; arrival rate 80% of the measured saturation throughput. Requests come from
    `clients` submitting threads (each a Poisson stream of rate/clients) and results are copied
    back to host memory by as many polling threads."""
    import numpy as np
    import torch

    import paper_1811_01201_gb300 as apsp
    from paper_1811_01201_gb300 import inputs
    ns = inputs.lognormal_sizes(pool_size, seed)
    pool = [inputs.dense_digraph(n, inputs.batch_graph_seed(seed, g), 1, 64).numpy() for g, n in enumerate(ns)]
    n_max = max(ns)

    def drive(srv, arrivals_per_client):
        jobs = [[] for _ in range(clients)]

        def client(ci, arrivals):
            t0 = start[0]
            for i, ta in enumerate(arrivals):
                dt = ta - (time.perf_counter() - t0)
                if dt > 0:
                    time.sleep(dt)
                W = pool[(ci * 7919 + i) % pool_size]
                jobs[ci].append((srv.submit(W), W.shape[0]))

        def poller(ci, total):
            k = 0
            outD = np.empty(n_max * n_max, np.float32)  # result buffers reused across jobs
            outP = np.empty(n_max * n_max, np.int32)
            while k < total:
                if k >= len(jobs[ci]):
                    time.sleep(0.0002)
                    continue
                jid, n = jobs[ci][k]
                srv.poll(jid, n, timeout_ms=-1, out=(outD[:n * n].reshape(n, n), outP[:n * n].reshape(n, n)))
                k += 1

        start = [time.perf_counter()]
        th = [threading.Thread(target=client, args=(c, arrivals_per_client[c])) for c in range(clients)]
        th += [threading.Thread(target=poller, args=(c, len(arrivals_per_client[c]))) for c in range(clients)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        return time.perf_counter() - start[0], sum(len(j) for j in jobs)

    budget = 100 << 30
    with apsp.Server(budget, max_slots=512) as srv:   # saturation: every request at time 0
        el, cnt = drive(srv, [[0.0] * 256 for _ in range(clients)])
        sat = cnt / el
    rate = 0.8 * sat
    count = max(clients, int(rate * seconds))
    per = count // clients
    arr = [inputs.poisson_arrivals(per, seed * 100 + c, rate / clients) for c in range(clients)]
    with apsp.Server(budget, max_slots=512) as srv:
        el, cnt = drive(srv, arr)
        st = srv.stats()
    flops = sum(2.0 * pool[(c * 7919 + i) % pool_size].shape[0] ** 3 for c in range(clients) for i in range(per))
    sweep = []
    for frac in (sweep_fracs or ()):
        # the same stream at other arrival rates (fractions of the measured saturation), shorter runs
        r_x = frac * sat
        per_x = max(1, int(r_x * sweep_seconds) // clients)
        arr_x = [inputs.poisson_arrivals(per_x, seed * 100 + 50 + c, r_x / clients) for c in range(clients)]
        with apsp.Server(budget, max_slots=512) as srv:
            el_x, cnt_x = drive(srv, arr_x)
            st_x = srv.stats()
        sweep.append({"load": frac, "arrival_rate_per_s": round(r_x, 1), "graphs_per_s": round(cnt_x / el_x, 1),
                      "p50_ms": round(st_x.p50_ms, 3), "p99_ms": round(st_x.p99_ms, 3),
                      "max_ms": round(st_x.max_ms, 3), "seconds": round(el_x, 2)})
    # the same request mix solved one at a time through the single-graph host call
    seq_n = min(64, pool_size)
    bufD = torch.empty(n_max * n_max)
    bufP = torch.empty(n_max * n_max, dtype=torch.int32)
    t0 = time.perf_counter()
    for i in range(seq_n):
        W = torch.from_numpy(pool[i])
        n = W.shape[0]
        apsp.apsp_fw_host(W, bufD[:n * n].view(n, n), bufP[:n * n].view(n, n))
    seq_gps = seq_n / (time.perf_counter() - t0)
    return {"workload": "Poisson requests, n=clip(round(lognormal(ln256,1)),32,4096), int weights U[1,64], "
                        f"100 GiB HBM budget, {clients} client threads; results copied to host on poll",
            "seconds": round(el, 2), "requests": cnt, "arrival_rate_per_s": round(rate, 1),
            "saturation_graphs_per_s": round(sat, 1), "graphs_per_s": round(cnt / el, 1),
            "gflops": round(flops / el / 1e9, 1), "p50_ms": round(st.p50_ms, 3), "p99_ms": round(st.p99_ms, 3),
            "max_ms": round(st.max_ms, 3), "hbm_peak_gib": round(st.hbm_peak / 2 ** 30, 3),
            "one_at_a_time_graphs_per_s": round(seq_gps, 1),
            **({"load_sweep": sweep} if sweep else {}),
            "speedup_vs_one_at_a_time": round(sat / seq_gps, 2)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=32768)
    ap.add_argument("--bs", type=int, default=64)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--kind", default="int", choices=["int", "real"],
                    help="weights: integer U[1,1000] (default) or real U(0,1]")
    ap.add_argument("--no-u16", dest="u16", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--paths", type=int, default=1 << 20, help="pairs for the apsp_paths line (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-sample-n", type=int, default=2560)
    ap.add_argument("--ref-sample-n", type=int, default=1536)
    ap.add_argument("--cpu-par-sample-n", type=int, default=6144)
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-extra-solves", dest="extra_solves", action="store_false",
                    help="skip the n=512, n=32768 real-weight and improving 16-bit solves")
    ap.add_argument("--no-c2", dest="autotune_c2", action="store_false",
                    help="skip the n=8192 density-0.5 solve with the autotuned block size")
    ap.add_argument("--workload", default="solve", choices=["solve", "batched", "serve"],
                    help="solve: the n=32768 single-graph line (with batched/served extras); "
                         "batched / serve: only that workload, as its own JSON line")
    ap.add_argument("--batch-count", type=int, default=4096, help="graphs of --workload batched")
    ap.add_argument("--batch-n", type=int, default=0, help="--workload batched: every graph of this order "
                    "(0: n log-uniform in [16,512])")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-sweep", action="store_true",
                    help="with --workload serve: also 15 s runs at 50%%, 95%% and 110%% of saturation")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "gb300" else args.warmup

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    if world > 1:
        import torch.distributed as dist
        if args.impl == "gb300":
            import torch
            torch.cuda.set_device(_env_int("LOCAL_RANK", 0))
            dist.init_process_group("nccl")
        else:
            dist.init_process_group("gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "solve":
        run_gpu(args, rank, world)
    else:
        run_extra(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
