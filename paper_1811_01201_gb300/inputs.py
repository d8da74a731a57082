"""Seeded synthetic inputs: dense random weighted digraphs.

This module only draws inputs; it holds none of the shortest-path arithmetic.
Both the CUDA library's tests/benchmarks and the CPU oracle's checks take
their graphs from here, so the two sides see bit-identical weights.

Every weight is a pure function of (seed, stream, element index), computed
with the SplitMix64 output function (Steele, Lea and Flood, "Fast Splittable
Pseudorandom Number Generators", OOPSLA 2014) on int64 tensors. The same
code therefore gives the same matrix on the CPU and on a GPU, in one piece or
in row slabs, so a sampled row of an n=32768 graph can be rebuilt on the host.

The paper measures on "workloads N" without naming a graph family
(Section 5.1); dense random weighted digraphs stand in for them.
"""

from __future__ import annotations

import math

import torch

_MASK64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15
_M1 = 0xBF58476D1CE4E5B9
_M2 = 0x94D049BB133111EB


def _signed(x: int) -> int:
    x &= _MASK64
    return x - (1 << 64) if x >= (1 << 63) else x


def mix64_int(x: int) -> int:
    """SplitMix64 output function on a Python int (reference, exact uint64)."""
    z = x & _MASK64
    z = ((z ^ (z >> 30)) * _M1) & _MASK64
    z = ((z ^ (z >> 27)) * _M2) & _MASK64
    return z ^ (z >> 31)


def _lsr(z: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of int64 lanes."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def mix64(z: torch.Tensor) -> torch.Tensor:
    """SplitMix64 output function on int64 lanes (two's-complement wraparound)."""
    z = (z ^ _lsr(z, 30)) * _signed(_M1)
    z = (z ^ _lsr(z, 27)) * _signed(_M2)
    return z ^ _lsr(z, 31)


def _stream_base(seed: int, stream: int) -> int:
    return mix64_int((seed * 256 + stream + 1) * _GAMMA)


def uniform24(seed: int, stream: int, idx: torch.Tensor) -> torch.Tensor:
    """24-bit uniform integers in [0, 2^24) for int64 element indices ``idx``."""
    base = _stream_base(seed, stream)
    z = mix64(idx.to(torch.int64) * _signed(_GAMMA) + _signed(base + _GAMMA))
    return _lsr(z, 40)


STREAM_WEIGHT = 0
STREAM_EDGE = 1
STREAM_PAIR = 2


def vertex_pairs(count: int, n: int, seed: int, device="cpu") -> torch.Tensor:
    """``count`` seeded (i, j) vertex pairs, uniform over [0, n)^2, as a (count, 2) int32 tensor."""
    u = uniform24(seed, STREAM_PAIR, torch.arange(2 * count, dtype=torch.int64, device=device))
    return ((u * n) >> 24).to(torch.int32).view(count, 2).contiguous()


def dense_digraph(n: int, seed: int, lo: float = 1, hi: float = 100, density: float = 1.0, kind: str = "int",
                  device="cpu", rows: tuple[int, int] | None = None, slab: int = 2048) -> torch.Tensor:
    """Weight matrix W (fp32, row-major n x n, or rows [r0, r1) of it).

    kind="int":  W[i][j] uniform integer in [lo, hi], stored as fp32.
    kind="real": W[i][j] uniform real in (0, 1], 24-bit resolution (1 - u).
    Each i != j edge is present with probability ``density`` (else +INF);
    W[i][i] = 0.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    r0, r1 = (0, n) if rows is None else rows
    out = torch.empty((r1 - r0, n), dtype=torch.float32, device=device)
    thresh = int(round(density * (1 << 24)))
    span = int(hi) - int(lo) + 1
    for s0 in range(r0, r1, slab):
        s1 = min(r1, s0 + slab)
        i = torch.arange(s0, s1, dtype=torch.int64, device=device).view(-1, 1)
        j = torch.arange(n, dtype=torch.int64, device=device).view(1, -1)
        idx = i * n + j
        u = uniform24(seed, STREAM_WEIGHT, idx)
        if kind == "int":
            w = (int(lo) + ((u * span) >> 24)).to(torch.float32)
        elif kind == "real":
            w = ((1 << 24) - u).to(torch.float32) * (1.0 / (1 << 24))
        else:
            raise ValueError(f"unknown kind {kind!r}")
        if density < 1.0:
            e = uniform24(seed, STREAM_EDGE, idx)
            w = torch.where(e < thresh, w, torch.full_like(w, math.inf))
        w = torch.where(i == j, torch.zeros_like(w), w)
        out[s0 - r0:s1 - r0] = w
    return out


def batch_sizes(count: int, seed: int, n_lo: int = 16, n_hi: int = 512) -> list[int]:
    """Graph orders n_g = round(exp(U(ln n_lo, ln n_hi))) (log-uniform)."""
    u = uniform24(seed, 2, torch.arange(count, dtype=torch.int64)).to(torch.float64) / (1 << 24)
    lo, hi = math.log(n_lo), math.log(n_hi)
    return [int(min(n_hi, max(n_lo, round(math.exp(lo + (hi - lo) * float(x)))))) for x in u]


def batch_graph_seed(seed: int, g: int) -> int:
    """Seed of graph g inside a seeded batch."""
    return seed * (1 << 20) + g + 1


def lognormal_sizes(count: int, seed: int, median: float = 256.0, sigma: float = 1.0, n_lo: int = 32,
                    n_hi: int = 4096) -> list[int]:
    """n = clip(round(lognormal(ln median, sigma)), n_lo, n_hi) via Box-Muller."""
    idx = torch.arange(count, dtype=torch.int64)
    u1 = (uniform24(seed, 3, idx).to(torch.float64) + 1.0) / ((1 << 24) + 1)
    u2 = uniform24(seed, 4, idx).to(torch.float64) / (1 << 24)
    z = torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)
    n = torch.exp(math.log(median) + sigma * z)
    return [int(min(n_hi, max(n_lo, round(float(x))))) for x in n]


def poisson_arrivals(count: int, seed: int, rate: float) -> list[float]:
    """Arrival times (s) of a Poisson process with the given rate (1/s)."""
    idx = torch.arange(count, dtype=torch.int64)
    u = (uniform24(seed, 5, idx).to(torch.float64) + 1.0) / ((1 << 24) + 1)
    gaps = -torch.log(u) / rate
    return torch.cumsum(gaps, 0).tolist()
