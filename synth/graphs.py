"""Seeded synthetic graph generators.

These graphs stand in for the social, web and road networks the paper
measures on (Section 5, Table 1: Facebook, Orkut, LiveJournal, Twitter,
Friendster, Road-CA/PA ...), none of which is available offline.  Every
generator is deterministic in its seed and returns a *canonical* CSR:
symmetric, loop-free, deduplicated, with each adjacency list sorted
ascending.  Node ids are ``uint32``; ``row_ptr`` is ``int64[n+1]``.

This module holds no part of the colour-coding method: it only makes
inputs.  Both the CPU oracle's tests and the CUDA path's tests and
benchmark draw their graphs from here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class CSRGraph:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # uint32[2m]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def neighbors(self, v: int) -> np.ndarray:
        return self.col[self.row_ptr[v]:self.row_ptr[v + 1]]


def from_edges(n: int, src, dst, name: str = "") -> CSRGraph:
    """Canonical CSR from an undirected edge list (any order, duplicates,
    self-loops and both orientations allowed)."""
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    if src.size:
        if src.min() < 0 or dst.min() < 0 or max(src.max(), dst.max()) >= n:
            raise ValueError("edge endpoint out of range")
    keep = src != dst
    src, dst = src[keep], dst[keep]
    a = np.concatenate([src, dst])
    b = np.concatenate([dst, src])
    key = a * np.int64(n) + b
    key.sort()
    if key.size:
        key = key[np.concatenate([[True], key[1:] != key[:-1]])]
    a = key // n
    b = key % n
    counts = np.bincount(a, minlength=n).astype(np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSRGraph(n=n, row_ptr=row_ptr, col=b.astype(np.uint32), name=name)


def relabel(g: CSRGraph, perm: np.ndarray) -> CSRGraph:
    """Rename node v to perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    dst = g.col.astype(np.int64)
    return from_edges(g.n, perm[src], perm[dst], name=g.name)


# --------------------------------------------------------------------------
# deterministic small graphs
# --------------------------------------------------------------------------

def path(n: int) -> CSRGraph:
    i = np.arange(n - 1)
    return from_edges(n, i, i + 1, name=f"path{n}")


def cycle(n: int) -> CSRGraph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, name=f"cycle{n}")


def star(leaves: int) -> CSRGraph:
    """Centre 0 joined to nodes 1..leaves."""
    i = np.arange(1, leaves + 1)
    return from_edges(leaves + 1, np.zeros_like(i), i, name=f"star{leaves}")


def clique(n: int) -> CSRGraph:
    a, b = np.triu_indices(n, 1)
    return from_edges(n, a, b, name=f"K{n}")


def lollipop(clique_size: int, tail: int) -> CSRGraph:
    """Clique on nodes 0..clique_size-1, plus a path of ``tail`` nodes
    hanging off node clique_size-1 (the lower-bound graph of Section 4.3.2)."""
    a, b = np.triu_indices(clique_size, 1)
    t = np.arange(clique_size - 1, clique_size + tail - 1)
    src = np.concatenate([a, t])
    dst = np.concatenate([b, t + 1])
    return from_edges(clique_size + tail, src, dst,
                      name=f"lollipop{clique_size}_{tail}")


def grid_road(side: int, seed: int = 0, p_delete: float = 0.10,
              p_diag: float = 0.02) -> CSRGraph:
    """Road-like planar graph: side x side grid, a fraction of grid edges
    deleted, a few diagonals added (max degree <= 8)."""
    rng = np.random.default_rng(seed)
    idx = np.arange(side * side, dtype=np.int64).reshape(side, side)
    h = np.stack([idx[:, :-1].ravel(), idx[:, 1:].ravel()])
    v = np.stack([idx[:-1, :].ravel(), idx[1:, :].ravel()])
    e = np.concatenate([h, v], axis=1)
    e = e[:, rng.random(e.shape[1]) >= p_delete]
    d = np.stack([idx[:-1, :-1].ravel(), idx[1:, 1:].ravel()])
    d = d[:, rng.random(d.shape[1]) < p_diag]
    e = np.concatenate([e, d], axis=1)
    return from_edges(side * side, e[0], e[1], name=f"grid{side}")


# --------------------------------------------------------------------------
# random graphs
# --------------------------------------------------------------------------

def erdos_renyi(n: int, avg_degree: float, seed: int = 0) -> CSRGraph:
    """G(n, p) with p = avg_degree / (n - 1).

    For n <= 20000 every pair is an independent Bernoulli trial.  Above
    that the edge count is drawn from the exact binomial and the pairs
    uniformly (duplicates dropped), which differs from G(n, p) by
    O(m^2 / n^2) edges."""
    rng = np.random.default_rng(seed)
    p = avg_degree / max(n - 1, 1)
    if n <= 20000:
        a, b = np.triu_indices(n, 1)
        keep = rng.random(a.size) < p
        return from_edges(n, a[keep], b[keep], name=f"er{n}")
    pairs = n * (n - 1) // 2
    m = int(rng.binomial(pairs, p))
    a = rng.integers(0, n, size=m, dtype=np.int64)
    b = rng.integers(0, n, size=m, dtype=np.int64)
    return from_edges(n, a, b, name=f"er{n}")


def chung_lu(n: int, m: int, exponent: float, max_degree: float | None = None,
             seed: int = 0, shuffle: bool = True) -> CSRGraph:
    """Chung-Lu power-law graph.

    Node weights w_i = (i + i0)^(-1/(exponent-1)); i0 is chosen so that the
    heaviest node's expected degree is ``max_degree`` (default sqrt(2 m),
    the usual structural cut-off).  m edges are drawn with both endpoints
    i.i.d. proportional to w; self-loops and duplicates are dropped, so the
    realised edge count is slightly below m.  With ``shuffle`` the node ids
    are randomly permuted, so hubs are not clustered at small ids."""
    rng = np.random.default_rng(seed)
    alpha = 1.0 / (exponent - 1.0)
    if max_degree is None:
        max_degree = float(np.sqrt(2.0 * m))
    i = np.arange(n, dtype=np.float64)

    def top_degree(i0: float) -> float:
        w = (i + i0) ** (-alpha)
        return 2.0 * m * w[0] / w.sum()

    lo, hi = 1e-9, float(n)
    for _ in range(200):  # expected top degree decreases in i0
        mid = np.sqrt(lo * hi)
        if top_degree(mid) > max_degree:
            lo = mid
        else:
            hi = mid
    w = (i + hi) ** (-alpha)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    # 2m i.i.d. endpoints (searched in sorted order for speed), then paired
    # up by a random permutation, which keeps the pairs i.i.d.
    ab = np.searchsorted(cdf, np.sort(rng.random(2 * m)), side="right")
    ab = ab[rng.permutation(2 * m)]
    a, b = ab[:m], ab[m:]
    a = np.minimum(a, n - 1)
    b = np.minimum(b, n - 1)
    if shuffle:
        perm = rng.permutation(n)
        a, b = perm[a], perm[b]
    return from_edges(n, a, b, name=f"cl{n}")


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19,
         c: float = 0.19, seed: int = 0, shuffle: bool = True) -> CSRGraph:
    """R-MAT graph on 2^scale nodes with edge_factor * 2^scale generated
    edges (quadrant probabilities a, b, c, d = 1 - a - b - c), symmetrised,
    loops and duplicates removed."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m = edge_factor * n
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    chunk = 1 << 22
    for s0 in range(0, m, chunk):
        s1 = min(m, s0 + chunk)
        u = np.zeros(s1 - s0, dtype=np.int64)
        v = np.zeros(s1 - s0, dtype=np.int64)
        for bit in range(scale):
            r = rng.random(s1 - s0)
            right = (r >= a) & (r < a + b) | (r >= a + b + c)
            down = r >= a + b
            u |= down.astype(np.int64) << bit
            v |= right.astype(np.int64) << bit
        src[s0:s1] = u
        dst[s0:s1] = v
    if shuffle:
        perm = rng.permutation(n)
        src, dst = perm[src], perm[dst]
    return from_edges(n, src, dst, name=f"rmat{scale}")


def random_colors(n: int, k: int, seed: int) -> np.ndarray:
    """An arbitrary caller-supplied colouring (uint8 in [0, k)), independent
    of the library's own counter-based colouring."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, k, size=n, dtype=np.uint8)


# --------------------------------------------------------------------------
# named workloads (the paper's graph families at the sizes we measure)
# --------------------------------------------------------------------------

def er_1k() -> CSRGraph:
    """Erdos-Renyi G(n=1000, p=8/999), seed 0."""
    return erdos_renyi(1000, 8.0, seed=0)


def chung_lu_1m() -> CSRGraph:
    """Chung-Lu n=1M, m~10M, degree exponent 2.5, max expected degree 10k."""
    return chung_lu(1_000_000, 10_000_000, 2.5, max_degree=10_000.0, seed=0)


def chung_lu_scaled(n: int, seed: int = 0) -> CSRGraph:
    """Same family as chung_lu_1m at n nodes (avg degree 20, exponent 2.5,
    max expected degree scaled as 10k * (n / 1M)^(1/1.5))."""
    md = 10_000.0 * (n / 1_000_000) ** (1.0 / 1.5)
    return chung_lu(n, 10 * n, 2.5, max_degree=max(md, 20.0), seed=seed)


def balanced_colors(n: int, k: int, seed: int) -> np.ndarray:
    """A caller colouring using every colour about n/k times (a random
    permutation of v mod k), so that tiny test graphs have colourful copies."""
    rng = np.random.default_rng(seed)
    return rng.permutation((np.arange(n) % k).astype(np.uint8))
