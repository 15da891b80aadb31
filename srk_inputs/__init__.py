"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only draws graphs, source lists and loss weights from fixed seeds.
It holds none of the SimRank method's arithmetic (no walk, table, shuffle or
score code), so both the CPU oracle and the CUDA library can take their inputs
from it without sharing any part of the computation.

Every graph is returned as an in-neighbour CSR: ``row_ptr`` (int32, n+1) and
``col`` (int32, m), where ``col[row_ptr[v]:row_ptr[v+1]]`` lists I(v), the
in-neighbours of v (the set used by Eq. 1 of the paper), sorted ascending,
without duplicates and without self-loops.

Recipes (the paper has no datasets; these stand in for its graphs):

* ``er_in_csr``: directed Erdos-Renyi.  For every node v an in-degree
  d ~ Poisson(mean) is drawn (capped at n-1) and d distinct in-neighbours are
  drawn uniformly from V minus {v}.
* ``rmat_in_csr``: R-MAT with 2**scale nodes and edge_factor * 2**scale edge
  draws.  Each draw descends ``scale`` levels of the adjacency matrix, choosing
  quadrant (row bit, column bit) = (0,0), (0,1), (1,0), (1,1) with
  probabilities (a, b, c, d) (one float32 uniform per level).  Row = source, column = target of the directed
  edge source -> target, so the source becomes an in-neighbour of the target.
  Self-loops are dropped, duplicates removed, node ids are not permuted.
* ``rmat_in_csr_torch``: the same R-MAT law drawn with torch's generator on a
  device (used for scale 22-24, where numpy takes minutes).
* ``uniform_sources``: distinct nodes drawn uniformly.
* ``mixed_sources`` / ``mixed_eps``: the batching workload's sources (a third
  of top in-degree, a third of median in-degree, a third without
  in-neighbours) and per-source eps drawn from {0.05, 0.02, 0.01}.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "er_in_csr",
    "rmat_in_csr",
    "uniform_sources",
    "mixed_sources",
    "lognormal_weights",
    "csr_from_edges",
    "rmat_in_csr_torch",
    "mixed_eps",
]


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray):
    """In-neighbour CSR of the directed edges src -> dst.

    Drops self-loops and duplicate edges; each in-list is sorted ascending.
    """
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    key = _sorted_unique(dst[keep] * n + src[keep])  # sorted by (dst, src), deduped
    dst_s = key // n
    col = (key - dst_s * n).astype(np.int32)
    counts = np.bincount(dst_s, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph has more than 2**31-1 edges")
    return row_ptr.astype(np.int32), col


def er_in_csr(n: int, mean_in_degree: float = 5.0, seed: int = 1):
    """Directed Erdos-Renyi graph with Poisson in-degrees (see module doc)."""
    if n < 1:
        raise ValueError("n must be positive")
    rng = np.random.default_rng(seed)
    degs = np.minimum(rng.poisson(mean_in_degree, size=n), n - 1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(degs, out=row_ptr[1:])
    col = np.empty(int(row_ptr[-1]), dtype=np.int32)
    for v in range(n):
        d = int(degs[v])
        if d == 0:
            continue
        pick = rng.choice(n - 1, size=d, replace=False)
        pick = np.where(pick >= v, pick + 1, pick)  # skip v itself
        col[row_ptr[v]:row_ptr[v + 1]] = np.sort(pick)
    return row_ptr.astype(np.int32), col


def _sorted_unique(key: np.ndarray) -> np.ndarray:
    key.sort()
    if key.size == 0:
        return key
    keep = np.empty(key.size, dtype=bool)
    keep[0] = True
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    return key[keep]


def rmat_in_csr(scale: int, edge_factor: int = 16,
                abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 1,
                chunk: int = 1 << 25):
    """R-MAT graph (see module doc), returned as an in-neighbour CSR.

    Each level draws one float32 uniform r per edge and picks the quadrant by
    the float32 thresholds a, a+b, a+b+c.
    """
    a, b, c, d = abcd
    if abs(a + b + c + d - 1.0) > 1e-9:
        raise ValueError("R-MAT probabilities must sum to 1")
    n = 1 << scale
    n_draws = edge_factor * n
    rng = np.random.default_rng(seed)
    t_a, t_ab, t_abc = np.float32(a), np.float32(a + b), np.float32(a + b + c)
    keys = []
    done = 0
    while done < n_draws:
        e = min(chunk, n_draws - done)
        src = np.zeros(e, dtype=np.int64)
        dst = np.zeros(e, dtype=np.int64)
        for level in range(scale):
            r = rng.random(e, dtype=np.float32)
            sh = scale - 1 - level
            row = r >= t_ab
            colb = ((r >= t_a) & (r < t_ab)) | (r >= t_abc)
            src += row.astype(np.int64) << sh
            dst += colb.astype(np.int64) << sh
        keep = src != dst
        keys.append(_sorted_unique(dst[keep] * n + src[keep]))
        done += e
    key = _sorted_unique(np.concatenate(keys)) if len(keys) > 1 else keys[0]
    dst_s = key >> scale
    col = (key & (n - 1)).astype(np.int32)
    counts = np.bincount(dst_s, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    if row_ptr[-1] > np.iinfo(np.int32).max:
        raise ValueError("graph has more than 2**31-1 edges")
    return row_ptr.astype(np.int32), col


def rmat_in_csr_torch(scale: int, edge_factor: int = 16,
                      abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 1,
                      device="cuda", chunk: int = 1 << 26):
    """The R-MAT recipe of ``rmat_in_csr`` drawn with torch's generator on
    ``device`` (fast for scale 22-24).  Same law, different random stream, so
    the graph differs from ``rmat_in_csr`` with the same seed.  Returns int32
    torch tensors (row_ptr, col) on ``device``."""
    import torch
    a, b, c, d = abcd
    n = 1 << scale
    n_draws = edge_factor * n
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    t_a, t_ab, t_abc = float(a), float(a + b), float(a + b + c)
    keys = []
    done = 0
    while done < n_draws:
        e = min(chunk, n_draws - done)
        src = torch.zeros(e, dtype=torch.int64, device=device)
        dst = torch.zeros(e, dtype=torch.int64, device=device)
        for level in range(scale):
            r = torch.rand(e, generator=gen, device=device, dtype=torch.float32)
            sh = scale - 1 - level
            src += (r >= t_ab).to(torch.int64) << sh
            dst += (((r >= t_a) & (r < t_ab)) | (r >= t_abc)).to(torch.int64) << sh
        keep = src != dst
        keys.append(torch.unique(dst[keep] * n + src[keep]))
        del src, dst, keep
        done += e
    key = torch.unique(torch.cat(keys)) if len(keys) > 1 else keys[0]
    del keys
    dst_s = key >> scale
    col = (key & (n - 1)).to(torch.int32)
    counts = torch.bincount(dst_s, minlength=n)
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(counts, 0)
    if int(row_ptr[-1]) > np.iinfo(np.int32).max:
        raise ValueError("graph has more than 2**31-1 edges")
    return row_ptr.to(torch.int32), col


def mixed_eps(k: int, seed: int = 3, choices=(0.05, 0.02, 0.01)) -> np.ndarray:
    """Per-source error targets drawn uniformly from ``choices``."""
    rng = np.random.default_rng(seed + 1000)
    return rng.choice(np.asarray(choices, dtype=np.float64), size=k)


def uniform_sources(n: int, k: int, seed: int = 2) -> np.ndarray:
    """k distinct source nodes drawn uniformly from [0, n)."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int32)


def mixed_sources(row_ptr: np.ndarray, k: int, seed: int = 3) -> np.ndarray:
    """k sources: a third of top in-degree, a third of median in-degree and the
    rest of zero in-degree nodes (drawn uniformly inside each group)."""
    deg = np.diff(row_ptr.astype(np.int64))
    n = deg.size
    rng = np.random.default_rng(seed)
    order = np.argsort(-deg, kind="stable")
    k_top = k // 3
    k_med = k // 3
    k_zero = k - k_top - k_med
    top = order[:max(k_top, 1) * 4]
    pos = np.flatnonzero(deg > 0)
    med_val = np.median(deg[pos]) if pos.size else 0
    med = np.flatnonzero(deg == int(med_val))
    zero = np.flatnonzero(deg == 0)
    out = []
    for group, cnt in ((top, k_top), (med, k_med), (zero, k_zero)):
        if cnt == 0:
            continue
        if group.size == 0:
            group = np.arange(n)
        out.append(rng.choice(group, size=cnt, replace=group.size < cnt))
    return np.concatenate(out).astype(np.int32)


def lognormal_weights(m: int, seed: int = 4, sigma: float = 0.5) -> np.ndarray:
    """FP32 edge weights ~ lognormal(0, sigma)."""
    rng = np.random.default_rng(seed)
    return rng.lognormal(0.0, sigma, size=m).astype(np.float32)
