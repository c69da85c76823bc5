"""Pins for round skipping and star sampling (Section 3.3.2) in the oracle.

* The balanced decomposition: both parts have at most k-2 nodes, they
  rebuild the shape, beta counts the equal root children; a_j (rooted
  copies per copy of tree j) recomputed by cutting edges, 0 exactly for the
  star (the lemma), k-2 for the path.
* Tables: level k holds the brute-force colourful rooted counts of every
  shape with a balanced decomposition and 0 elsewhere; level k-1 is absent;
  the unrooted totals equal those of the full build for every non-star tree.
* The sampler draws each colourful non-star copy of tree j with probability
  a_j / R (exact distribution by brute force, chi-square).
* The star sampler is uniform over the h-stars of the graph (centre and
  leaf set), whose number is sum_v C(d_v, h-1).
* Estimates: unbiased for every graphlet, the star-only graphlet from the
  uncoloured stars.
"""
import itertools
import math
from collections import Counter

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import brute
from tests.test_oracle_sampling import _chi2_ok


def _cut_rootings(adj, k):
    """Nodes x with a neighbour y whose side of the edge xy has 2..k-2 nodes."""
    def side(y, x):
        seen, stack = {y}, [y]
        while stack:
            a = stack.pop()
            for b in adj[a]:
                if b != x and b not in seen:
                    seen.add(b)
                    stack.append(b)
        return len(seen)
    return sum(1 for x in adj if any(2 <= side(y, x) <= k - 2 for y in adj[x]))


@pytest.mark.parametrize("k", range(4, 9))
def test_balanced_decomposition(k):
    for s in cat.rooted_shapes(k):
        d = cat.balanced_decompose(s, k)
        kids = cat._split_children(s)
        sizes = [len(c) // 2 for c in kids]
        if d is None:
            assert all(z in (1, k - 1) for z in sizes)
            continue
        a, b, beta = d
        na, nb = len(a) // 2 + 1, len(b) // 2 + 1
        assert na + nb == k and 2 <= nb <= k - 2 and na <= k - 2
        assert cat.canonical_from_children([c[1:-1] for c in cat._split_children(a)] + [b]) == s
        assert beta == kids.count("1" + b + "0")
        assert a in cat.rooted_shapes(na) and b in cat.rooted_shapes(nb)
    C = cat.Catalog(k, skip_round=True)
    star = cat.unrooted_id("10" * (k - 1))
    path = cat.unrooted_id(cat.encode(cat.decode("1" * (k - 1) + "0" * (k - 1)), 0))
    for j, (code, a_j) in enumerate(zip(cat.unrooted_shapes(k), C.copies_divisor(k))):
        adj = cat.decode(format(code, "0%db" % (2 * (k - 1))))
        assert a_j == _cut_rootings(adj, k)
        assert (a_j == 0) == (j == star)
    assert C.copies_divisor(k)[path] == k - 2


def _table_dict(T, h, C):
    lv = T.level_int(h)
    masks = [m for m in range(1 << T.k) if bin(m).count("1") == h]
    out = {}
    for v in range(T.n):
        for s_i, s in enumerate(cat.rooted_shapes(h)):
            for q, m in enumerate(masks):
                if lv[v][s_i][q]:
                    out[(v, s, m)] = lv[v][s_i][q]
    return out


@pytest.mark.parametrize("k", [4, 5, 6])
def test_skip_tables_match_brute_force(oracle, k):
    graphs = [synth.erdos_renyi(9, 4.0, seed=k), synth.clique(7), synth.lollipop(5, 3),
              synth.grid_road(3, seed=1, p_diag=0.5)]
    for gi, g in enumerate(graphs):
        colors = synth.random_colors(g.n, k, seed=20 + gi)
        Z = oracle.Tables(g, colors, k, 128, nthreads=2, skip_round=True)
        A = oracle.Tables(g, colors, k, 128, nthreads=2)
        counted = {s for s in cat.rooted_shapes(k) if cat.balanced_decompose(s, k) is not None}
        want = {key: c for key, c in brute.treelet_counts(g, colors, k).items() if key[1] in counted}
        assert _table_dict(Z, k, counted) == want, (g.name, k)
        for h in range(1, k - 1):
            assert np.array_equal(Z.level(h), A.level(h))
        with pytest.raises(oracle.OracleError):
            Z.level(k - 1)
        star = cat.unrooted_id("10" * (k - 1))
        for j in range(len(cat.unrooted_shapes(k))):
            assert Z.total(k, j)[1] == (0 if j == star else A.total(k, j)[1])
        assert Z.total(k)[1] == A.total(k)[1] - A.total(k, star)[1]


def _exact_skip_outcomes(g, colors, k):
    """{(sorted nodes, root, rooted shape id): numerator}, total: one unit per
    colourful spanning tree of a node set and balanced rooting of it."""
    adj = brute.adjacency(g)
    shapes = cat.rooted_shapes(k)
    out = Counter()
    for S in itertools.combinations(range(g.n), k):
        if len({int(colors[v]) for v in S}) != k:
            continue
        for tree in brute.spanning_trees(adj, S):
            ta = {v: [] for v in S}
            for a, b in tree:
                ta[a].append(b)
                ta[b].append(a)
            for r in S:
                s = cat.encode(ta, r)
                if cat.balanced_decompose(s, k) is not None:
                    out[(S, r, shapes.index(s))] += 1
    return out, sum(out.values())


@pytest.mark.parametrize("k,seed", [(4, 1), (5, 2)])
def test_skip_sampler_distribution(oracle, k, seed):
    g = synth.erdos_renyi(9, 4.5, seed=seed)
    colors = synth.balanced_colors(g.n, k, seed=seed)
    Z = oracle.Tables(g, colors, k, 64, nthreads=1, skip_round=True)
    exact, total = _exact_skip_outcomes(g, colors, k)
    assert total == Z.total(k)[0]
    N = 40 * len(exact) + 4000
    nodes, roots, shapes, _ = Z.sample(k, seed=3, first_index=0, count=N)
    obs = Counter((tuple(int(x) for x in nodes[i]), int(roots[i]), int(shapes[i]))
                  for i in range(N))
    assert _chi2_ok(obs, exact, total, N)
    with pytest.raises(oracle.OracleError):
        Z.sample(k - 1, seed=1, first_index=0, count=1)


@pytest.mark.parametrize("h", [3, 4, 5])
def test_star_sampler_is_uniform(oracle, h):
    g = synth.chung_lu(14, 30, 2.2, seed=h)
    colors = synth.random_colors(g.n, 5, seed=0)
    T = oracle.Tables(g, colors, 5, 64, nthreads=1)
    adj = brute.adjacency(g)
    stars = Counter()
    for v in range(g.n):
        for leaves in itertools.combinations(sorted(adj[v]), h - 1):
            stars[(tuple(sorted((v,) + leaves)), v)] += 1
    total = sum(stars.values())
    assert T.star_total(h) == total == sum(math.comb(len(adj[v]), h - 1) for v in range(g.n))
    N = 40 * len(stars) + 4000
    nodes, centres, classes = T.sample_stars(h, seed=9, first_index=0, count=N)
    obs = Counter((tuple(int(x) for x in nodes[i]), int(centres[i])) for i in range(N))
    assert _chi2_ok(obs, stars, total, N)
    for i in range(200):
        S = [int(x) for x in nodes[i]]
        assert classes[i] == oracle.class_of_word(h, brute.word_of(adj, S))
    a = T.sample_stars(h, seed=9, first_index=100, count=10)
    assert np.array_equal(a[0], nodes[100:110])


def test_skip_estimates_unbiased(oracle):
    k = 4
    g = synth.erdos_renyi(14, 5.0, seed=6)
    colors = synth.balanced_colors(g.n, k, seed=6)
    Z = oracle.Tables(g, colors, k, 64, skip_round=True)
    classify = lambda w: oracle.class_of_word(k, w)
    truth = brute.colourful_graphlets(g, colors, k, classify)
    every = brute.graphlets(g, k, classify)
    _, s_ij = oracle.sigma(k)
    a = np.asarray(cat.Catalog(k, True).copies_divisor(k), np.int64)
    s_prime = s_ij @ a
    star = cat.unrooted_id("10" * (k - 1))
    R = Z.total(k)[0]
    S = Z.star_total(k)
    N = 200_000
    est, hits = Z.estimate_uniform(k, seed=3, n_samples=N, star_samples=N)
    p = 1.0 / oracle.inv_colorful_prob(k, k)
    for i in range(len(s_prime)):
        if s_prime[i] > 0:
            c = truth.get(i, 0)
            q = c * int(s_prime[i]) / R
            sd = R / int(s_prime[i]) * math.sqrt(q * (1 - q) / N)
            assert abs(est[i] * p - c) <= 5 * sd + 1e-9, (i, est[i] * p, c)
        else:
            gi, ss = every.get(i, 0), int(s_ij[i, star])
            q = gi * ss / S
            sd = S / ss * math.sqrt(q * (1 - q) / N)
            assert abs(est[i] - gi) <= 5 * sd + 1e-9, (i, est[i], gi)
    # AGS: the star-only graphlet comes from the same star stream
    e2, h2, st = Z.estimate_ags(k, seed=3, max_samples=100_000, cbar=200, star_samples=N)
    star_only = np.flatnonzero(s_prime == 0)
    assert np.array_equal(e2[star_only], est[star_only])
    assert np.array_equal(h2[star_only], hits[star_only])
    target = int((s_prime > 0).sum())
    assert st["covered"] <= target and (st["covered"] == target or st["samples"] == 100_000)
    seen = [i for i in range(len(s_prime)) if s_prime[i] > 0 and truth.get(i, 0) > 0]
    assert all(h2[i] > 0 for i in seen)
