"""Brute-force enumerations on tiny graphs, used to pin the oracle.

Nothing here follows the paper's dynamic program: treelet copies are found
by listing node subsets and edge subsets and testing each one directly.
"""
from __future__ import annotations

import itertools
from collections import Counter

import numpy as np

from oracle import catalog as cat


def adjacency(g) -> list[set[int]]:
    return [set(int(x) for x in g.neighbors(v)) for v in range(g.n)]


def _is_spanning_tree(nodes, edges) -> bool:
    parent = {v: v for v in nodes}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in edges:
        ra, rb = find(a), find(b)
        if ra == rb:
            return False
        parent[ra] = rb
    return len(edges) == len(nodes) - 1


def induced_edges(adj, nodes) -> list[tuple[int, int]]:
    nodes = sorted(nodes)
    return [(a, b) for i, a in enumerate(nodes) for b in nodes[i + 1:] if b in adj[a]]


def spanning_trees(adj, nodes):
    """Every spanning tree of the induced subgraph, as an edge list."""
    es = induced_edges(adj, nodes)
    for sub in itertools.combinations(es, len(nodes) - 1):
        if _is_spanning_tree(nodes, sub):
            yield sub


def _tree_adj(nodes, edges):
    adj = {v: [] for v in nodes}
    for a, b in edges:
        adj[a].append(b)
        adj[b].append(a)
    return adj


def treelet_counts(g, colors, h) -> dict[tuple[int, str, int], int]:
    """{(v, s_T, colour mask): number of colourful copies of T_C rooted at v}
    for |T| = h, by listing node sets and their spanning trees."""
    adj = adjacency(g)
    out: Counter = Counter()
    for S in itertools.combinations(range(g.n), h):
        mask = 0
        for v in S:
            mask |= 1 << int(colors[v])
        if bin(mask).count("1") != h:
            continue
        for tree in spanning_trees(adj, S):
            ta = _tree_adj(S, tree)
            for v in S:
                out[(v, cat.encode(ta, v), mask)] += 1
    return dict(out)


def tree_copies(g, h) -> Counter:
    """{unrooted code: number of (non-induced) h-node subtrees of that shape}."""
    adj = adjacency(g)
    out: Counter = Counter()
    for S in itertools.combinations(range(g.n), h):
        for tree in spanning_trees(adj, S):
            ta = _tree_adj(S, tree)
            out[min(int(cat.encode(ta, r), 2) if h > 1 else 0 for r in S)] += 1
    return out


def is_connected(adj, nodes) -> bool:
    nodes = list(nodes)
    seen = {nodes[0]}
    stack = [nodes[0]]
    ns = set(nodes)
    while stack:
        x = stack.pop()
        for y in adj[x]:
            if y in ns and y not in seen:
                seen.add(y)
                stack.append(y)
    return len(seen) == len(nodes)


def word_of(adj, nodes) -> int:
    """Adjacency word of the induced subgraph on the sorted nodes: pairs
    (i, j), i < j, lexicographic, first pair most significant."""
    nodes = sorted(nodes)
    h = len(nodes)
    bits = [1 if nodes[j] in adj[nodes[i]] else 0 for i in range(h) for j in range(i + 1, h)]
    w = 0
    for b in bits:
        w = (w << 1) | b
    return w


def graph_of_word(h: int, w: int) -> list[set[int]]:
    pairs = [(i, j) for i in range(h) for j in range(i + 1, h)]
    P = len(pairs)
    adj = [set() for _ in range(h)]
    for p, (i, j) in enumerate(pairs):
        if (w >> (P - 1 - p)) & 1:
            adj[i].add(j)
            adj[j].add(i)
    return adj


def colourful_graphlets(g, colors, h, classify) -> Counter:
    """{class id: number of colourful induced connected h-node subgraphs}."""
    adj = adjacency(g)
    out: Counter = Counter()
    for S in itertools.combinations(range(g.n), h):
        if len({int(colors[v]) for v in S}) != h or not is_connected(adj, S):
            continue
        out[classify(word_of(adj, S))] += 1
    return out


def graphlets(g, h, classify) -> Counter:
    adj = adjacency(g)
    out: Counter = Counter()
    for S in itertools.combinations(range(g.n), h):
        if is_connected(adj, S):
            out[classify(word_of(adj, S))] += 1
    return out


def colour_counts(g, colors, k):
    """[n, k] neighbour counts per colour."""
    src = np.repeat(np.arange(g.n, dtype=np.int64), g.degrees())
    idx = src * k + colors[g.col.astype(np.int64)].astype(np.int64)
    return np.bincount(idx, minlength=g.n * k).reshape(g.n, k)


def star_totals(g, colors, k):
    """{h: number of colourful h-stars}, h = 2..k, as exact integers."""
    cnt = colour_counts(g, colors, k)
    cnt[np.arange(g.n), colors.astype(np.int64)] = 0      # neighbours of the centre's colour
    e = [np.ones(g.n, dtype=object)] + [np.zeros(g.n, dtype=object) for _ in range(k - 1)]
    for a in range(k):
        x = cnt[:, a].astype(object)
        for j in range(k - 1, 0, -1):
            e[j] = e[j] + e[j - 1] * x
    out = {2: int(e[1].sum()) // 2}
    for h in range(3, k + 1):
        out[h] = int(e[h - 1].sum())
    return out
