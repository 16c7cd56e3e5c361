"""Seeded synthetic graphs (the inputs of every test and benchmark).

This module holds none of SketchNE's arithmetic: it only draws undirected,
unweighted graphs with NumPy's PCG64 generator and returns them as symmetric
CSR arrays (both directions of every edge stored, columns sorted within each
row, no self-loops, no duplicate edges).  The oracle, the tests and the
benchmark all take their graphs from here, so that both sides of every parity
check see the same input.

Graph families (stand-ins for the paper's datasets of Table 1):

* ``sbm``: stochastic block model with equal blocks.  Every vertex pair is an
  edge independently with probability ``p_in`` (same block) or ``p_out``;
  drawn exactly in distribution as a binomial edge count per block pair
  followed by a uniform choice of that many distinct pairs.
* ``chung_lu``: power-law Chung-Lu graph.  Vertex weights
  ``w_i ~ (i + i0)^(-1/(gamma-1))`` are scaled so that their sum is
  ``n * avg_degree`` after capping every weight at ``sqrt(n * avg_degree)``;
  endpoint pairs are drawn i.i.d. with probability proportional to ``w``,
  self-loops and repeats are dropped, and drawing continues until at least
  ``n * avg_degree / 2`` distinct edges exist (the last batch of draws
  overshoots, so the realized mean degree is up to about 1% above the target).
  Vertex ids are therefore sorted by expected degree (id 0 is the largest hub).
* ``complete_graph``, ``complete_bipartite_union``, ``from_edges``: small
  graphs with closed-form spectra, used to pin the oracle.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass
class Graph:
    """Symmetric CSR: ``row_ptr`` int64 [n+1], ``col_idx`` int32 [nnz]."""

    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)


def _csr_from_undirected_pairs(n: int, i: np.ndarray, j: np.ndarray, name: str = "") -> Graph:
    """Build a symmetric CSR from undirected pairs (self-loops and repeats removed)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    keep = i != j
    i, j = i[keep], j[keep]
    key = np.unique(np.minimum(i, j) * n + np.maximum(i, j))
    return _csr_from_unique_keys(n, key, name)


def _csr_from_unique_keys(n: int, key: np.ndarray, name: str = "") -> Graph:
    """CSR from sorted unique keys lo*n + hi (lo < hi) of undirected edges."""
    lo = key // n
    hi = key - lo * n
    both = np.concatenate([key, hi * n + lo])
    both.sort()
    src = both // n
    dst = both - src * n
    counts = np.bincount(src, minlength=n)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return Graph(n=n, row_ptr=row_ptr, col_idx=dst.astype(np.int32), name=name)


def from_edges(n: int, edges, name: str = "") -> Graph:
    e = np.asarray(list(edges), dtype=np.int64).reshape(-1, 2)
    return _csr_from_undirected_pairs(n, e[:, 0], e[:, 1], name=name)


def complete_graph(n: int) -> Graph:
    i, j = np.triu_indices(n, k=1)
    return _csr_from_undirected_pairs(n, i, j, name=f"K{n}")


def complete_bipartite_union(parts) -> Graph:
    """Disjoint union of complete bipartite graphs K_{a,b}, one per (a, b) in ``parts``."""
    src, dst = [], []
    base = 0
    for a, b in parts:
        left = np.arange(base, base + a)
        right = np.arange(base + a, base + a + b)
        ii, jj = np.meshgrid(left, right, indexing="ij")
        src.append(ii.ravel())
        dst.append(jj.ravel())
        base += a + b
    return _csr_from_undirected_pairs(base, np.concatenate(src), np.concatenate(dst),
                                      name="Kab-union")


def _decode_triangle(idx: np.ndarray, m: int):
    """Map a linear index over the pairs (i < j) of an m-set to (i, j)."""
    idx = idx.astype(np.int64)
    # row i starts at s(i) = i*(2m - i - 1)/2
    b = 2 * m - 1
    i = np.floor((b - np.sqrt(np.maximum(b * b - 8.0 * idx, 0.0))) / 2.0).astype(np.int64)
    i = np.clip(i, 0, m - 2)

    def start(r):
        return r * (2 * m - r - 1) // 2

    # correct floating-point rounding of the square root
    for _ in range(3):
        i = np.where(start(i) > idx, i - 1, i)
        i = np.where(start(i + 1) <= idx, i + 1, i)
    j = idx - start(i) + i + 1
    return i, j


def sbm(n: int, blocks: int, p_in: float, p_out: float, seed: int = 0) -> Graph:
    rng = np.random.Generator(np.random.PCG64(seed))
    bounds = np.linspace(0, n, blocks + 1).round().astype(np.int64)
    src, dst = [], []
    for a in range(blocks):
        for b in range(a, blocks):
            na = bounds[a + 1] - bounds[a]
            nb = bounds[b + 1] - bounds[b]
            if a == b:
                npairs = na * (na - 1) // 2
                p = p_in
            else:
                npairs = na * nb
                p = p_out
            if npairs == 0 or p <= 0:
                continue
            cnt = int(rng.binomial(npairs, p))
            if cnt == 0:
                continue
            pick = rng.choice(npairs, size=cnt, replace=False)
            if a == b:
                ii, jj = _decode_triangle(pick, int(na))
            else:
                ii, jj = pick // nb, pick % nb
            src.append(ii + bounds[a])
            dst.append(jj + bounds[b])
    if not src:
        return _csr_from_undirected_pairs(n, np.zeros(0), np.zeros(0), name="sbm")
    return _csr_from_undirected_pairs(n, np.concatenate(src), np.concatenate(dst),
                                      name=f"sbm(n={n},B={blocks},pin={p_in},pout={p_out},seed={seed})")


def chung_lu(n: int, avg_degree: float, gamma: float, seed: int = 0, i0: float = 1.0,
             chunk: int = 1 << 24) -> Graph:
    rng = np.random.Generator(np.random.PCG64(seed))
    target = n * avg_degree
    # scaled so that sum(min(s * base, sqrt(sum))) = n * avg_degree (the cap keeps p_ij <= 1)
    w = chung_lu_weights(n, avg_degree, gamma, i0)
    cdf = np.cumsum(w / w.sum())
    cdf[-1] = 1.0
    want = int(round(target / 2.0))  # distinct undirected edges
    key = np.zeros(0, dtype=np.int64)
    draw = want
    while key.size < want:
        parts = []
        for c0 in range(0, draw, chunk):
            c = min(chunk, draw - c0)
            a = np.minimum(np.searchsorted(cdf, rng.random(c), side="right"), n - 1)
            b = np.minimum(np.searchsorted(cdf, rng.random(c), side="right"), n - 1)
            keep = a != b
            a, b = a[keep], b[keep]
            parts.append(np.minimum(a, b).astype(np.int64) * n + np.maximum(a, b))
        key = np.unique(np.concatenate([key, *parts]))
        draw = int((want - key.size) * 1.3) + 1024
    return _csr_from_unique_keys(n, key, name=f"chung_lu(n={n},avg={avg_degree},gamma={gamma},seed={seed})")


def chung_lu_weights(n: int, avg_degree: float, gamma: float, i0: float = 1.0) -> np.ndarray:
    """The vertex weights of ``chung_lu`` (power law, capped at sqrt(n avg))."""
    base = (np.arange(n, dtype=np.float64) + i0) ** (-1.0 / (gamma - 1.0))
    target = n * avg_degree
    cap = np.sqrt(target)
    lo_s, hi_s = 0.0, target / base.sum() * 1e3
    for _ in range(100):
        mid = 0.5 * (lo_s + hi_s)
        if np.minimum(base * mid, cap).sum() < target:
            lo_s = mid
        else:
            hi_s = mid
    return np.minimum(base * hi_s, cap)


def chung_lu_device(n: int, avg_degree: float, gamma: float, seed: int = 0, device="cuda",
                    chunk: int = 1 << 27):
    """The Chung-Lu recipe of ``chung_lu`` drawn on a GPU with torch's
    generator (seeded; a different stream of random numbers than the NumPy
    version, so a different graph from the same distribution), for graphs
    whose NumPy generation would take many minutes (n = 5 * 10^7, about
    2 * 10^9 stored entries).  Returns (row_ptr int64 [n+1], col_idx int32
    [nnz]) as device tensors, columns sorted within each row."""
    import torch
    w = torch.as_tensor(chung_lu_weights(n, avg_degree, gamma), dtype=torch.float64, device=device)
    cdf = torch.cumsum(w / w.sum(), 0)
    cdf[-1] = 1.0
    del w
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    want = int(round(n * avg_degree / 2.0))
    key = torch.zeros(0, dtype=torch.int64, device=device)
    draw = want
    while key.numel() < want:
        parts = [key]
        for c0 in range(0, draw, chunk):
            c = min(chunk, draw - c0)
            a = torch.searchsorted(cdf, torch.rand(c, generator=gen, device=device, dtype=torch.float64),
                                   right=True).clamp_(max=n - 1)
            b = torch.searchsorted(cdf, torch.rand(c, generator=gen, device=device, dtype=torch.float64),
                                   right=True).clamp_(max=n - 1)
            keep = a != b
            a, b = a[keep], b[keep]
            parts.append(torch.minimum(a, b) * n + torch.maximum(a, b))
            del a, b, keep
        key = torch.unique(torch.cat(parts))
        del parts
        draw = int((want - key.numel()) * 1.3) + 1024
    lo = key // n
    hi = key - lo * n
    del key
    both = torch.cat([lo * n + hi, hi * n + lo])
    del lo, hi
    both, _ = torch.sort(both)
    src = both // n
    col = (both - src * n).to(torch.int32)
    del both
    counts = torch.bincount(src, minlength=n)
    del src
    row_ptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=row_ptr[1:])
    return row_ptr, col


def batched_mix(count: int = 64, n_lo: int = 2000, n_hi: int = 200000, deg_lo: float = 8.0,
                deg_hi: float = 32.0, seed: int = 0):
    """Uneven batch of graphs: graph g is seeded g; even g -> 8-block SBM with
    p_in/p_out = 10, odd g -> Chung-Lu with gamma = 2.1."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    degs = rng.uniform(deg_lo, deg_hi, size=count)
    graphs = []
    for g in range(count):
        n = int(ns[g])
        avg = float(degs[g])
        if g % 2 == 0:
            blk = n / 8.0
            p_out = avg / (17.0 * blk)
            graphs.append(sbm(n, 8, 10.0 * p_out, p_out, seed=g))
        else:
            graphs.append(chung_lu(n, avg, 2.1, seed=g))
    return graphs


def named(config: str) -> Graph:
    """The graph of a named workload."""
    if config == "sbm4096":
        return sbm(4096, 8, 0.01, 0.001, seed=0)
    if config == "cl1m":
        return chung_lu(1_000_000, 20.0, 2.1, seed=0)
    if config == "cl10m":
        return chung_lu(10_000_000, 30.0, 2.2, seed=0)
    raise KeyError(config)
