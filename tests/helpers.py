"""Shared test helpers: golden-fixture parsing and a brute-force APSP."""

from __future__ import annotations

import math
import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _num(tok: str) -> float:
    return math.inf if tok == "inf" else float(tok)


def load_golden(name: str) -> dict:
    """Parse a tests/golden/*.txt fixture into a dict of numpy arrays."""
    out: dict = {}
    key = None
    rows: list = []
    with open(os.path.join(GOLDEN, name)) as f:
        lines = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    for ln in lines:
        parts = ln.split()
        if parts[0] in ("n", "bs"):
            out[parts[0]] = int(parts[1])
            continue
        if len(parts) == 1 and not parts[0].lstrip("-").replace(".", "").isdigit() and parts[0] != "inf":
            if key is not None:
                out[key] = rows
            key, rows = parts[0], []
            continue
        rows.append([_num(t) for t in parts])
    if key is not None:
        out[key] = rows
    for k, v in list(out.items()):
        if isinstance(v, list):
            arr = np.array(v, dtype=np.float64)
            out[k] = arr.astype(np.int32) if k.startswith("P") else arr.astype(np.float32)
    return out


def brute_force_apsp(W: np.ndarray) -> np.ndarray:
    """Exact shortest distances by enumerating every simple path (n <= 7)."""
    n = W.shape[0]
    assert n <= 7
    D = np.full((n, n), math.inf)
    w = W.astype(np.float64)

    def dfs(src, u, cost, seen):
        if cost < D[src][u]:
            D[src][u] = cost
        for v in range(n):
            if v not in seen and math.isfinite(w[u][v]) and v != u:
                seen.add(v)
                dfs(src, v, cost + w[u][v], seen)
                seen.discard(v)

    for s in range(n):
        dfs(s, s, 0.0, {s})
    return D


def all_pairs(n: int) -> np.ndarray:
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    return np.stack([ii.ravel(), jj.ravel()], axis=1).astype(np.int32)


def random_pairs(n: int, count: int, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, size=(count, 2)).astype(np.int32)
