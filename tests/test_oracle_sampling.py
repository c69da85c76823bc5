"""Pins for the oracle's sampler and estimators (Section 2.2, Section 4.1).

The sampler is checked against the exact distribution it must follow: each
colourful h-treelet copy with probability 1/t, each of its h rootings
equally likely.  The exact distribution is found by brute force (node sets
and their spanning trees); the empirical one by seeded sampling; chi-square
compares them.  The estimators are checked for unbiasedness against
brute-force colourful graphlet counts, and AGS against its (1 +- eps)
guarantee (Theorem 3).
"""
import math
from collections import Counter

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import brute


def _exact_outcomes(g, colors, h, unrooted=None):
    """{(sorted nodes, root, rooted shape id): probability numerator}, total."""
    adj = brute.adjacency(g)
    shapes = cat.rooted_shapes(h)
    out = Counter()
    import itertools
    for S in itertools.combinations(range(g.n), h):
        if len({int(colors[v]) for v in S}) != h:
            continue
        for tree in brute.spanning_trees(adj, S):
            ta = {v: [] for v in S}
            for a, b in tree:
                ta[a].append(b)
                ta[b].append(a)
            if unrooted is not None:
                code = min(int(cat.encode(ta, r), 2) for r in S)
                if cat.unrooted_shapes(h).index(code) != unrooted:
                    continue
            for r in S:
                out[(S, r, shapes.index(cat.encode(ta, r)))] += 1
    return out, sum(out.values())


def _chi2_ok(observed: Counter, expected_num: Counter, total: int, N: int) -> bool:
    assert set(observed) <= set(expected_num), "sample outside the support"
    chi2 = 0.0
    for key, num in expected_num.items():
        e = N * num / total
        chi2 += (observed.get(key, 0) - e) ** 2 / e
    dof = len(expected_num) - 1
    return chi2 < dof + 6.0 * math.sqrt(2.0 * dof)


@pytest.mark.parametrize("k,seed", [(3, 1), (4, 2), (5, 3), (6, 4)])
def test_sampler_is_uniform_over_colourful_treelets(oracle, k, seed):
    g = synth.erdos_renyi(9, 4.0, seed=seed)
    colors = synth.balanced_colors(g.n, k, seed=seed)
    T = oracle.Tables(g, colors, k, 64, nthreads=1)
    exact, total = _exact_outcomes(g, colors, k)
    assert total == T.total(k)[0]
    N = 40 * len(exact) + 4000
    nodes, roots, shapes, _ = T.sample(k, seed=11, first_index=0, count=N)
    obs = Counter((tuple(int(x) for x in nodes[i]), int(roots[i]), int(shapes[i]))
                  for i in range(N))
    assert _chi2_ok(obs, exact, total, N)


def test_zero_rooted_sampler_is_uniform(oracle):
    # with zero-rooting the root is each copy's colour-0 node; every colourful
    # k-treelet copy must still come up with probability 1/t
    k = 4
    g = synth.erdos_renyi(10, 4.5, seed=12)
    colors = synth.balanced_colors(g.n, k, seed=12)
    T = oracle.Tables(g, colors, k, 64, nthreads=1, zero_root=True)
    exact, total = _exact_outcomes(g, colors, k)
    exact = Counter({key: c for key, c in exact.items() if colors[key[1]] == 0})
    total = sum(exact.values())
    assert total == T.total(k)[0] == T.total(k)[1]
    N = 40 * len(exact) + 4000
    nodes, roots, shapes, _ = T.sample(k, seed=3, first_index=0, count=N)
    obs = Counter((tuple(int(x) for x in nodes[i]), int(roots[i]), int(shapes[i]))
                  for i in range(N))
    assert _chi2_ok(obs, exact, total, N)


def test_sampler_restricted_to_one_shape(oracle):
    k = 4
    g = synth.erdos_renyi(10, 4.5, seed=4)
    colors = synth.balanced_colors(g.n, k, seed=4)
    T = oracle.Tables(g, colors, k, 64, nthreads=1)
    for j in range(len(cat.unrooted_shapes(k))):
        exact, total = _exact_outcomes(g, colors, k, unrooted=j)
        assert total == T.total(k, j)[0]
        N = 40 * len(exact) + 2000
        nodes, roots, shapes, _ = T.sample(k, seed=5, first_index=0, count=N, unrooted=j)
        obs = Counter((tuple(int(x) for x in nodes[i]), int(roots[i]), int(shapes[i]))
                      for i in range(N))
        assert _chi2_ok(obs, exact, total, N)


def test_sampler_smaller_h_than_k(oracle):
    # h-treelets drawn from tables built with k > h colours
    k, h = 5, 3
    g = synth.erdos_renyi(9, 4.0, seed=8)
    colors = synth.balanced_colors(g.n, k, seed=8)
    T = oracle.Tables(g, colors, k, 64, nthreads=1)
    exact, total = _exact_outcomes(g, colors, h)
    N = 40 * len(exact) + 2000
    nodes, roots, shapes, _ = T.sample(h, seed=2, first_index=0, count=N)
    obs = Counter((tuple(int(x) for x in nodes[i]), int(roots[i]), int(shapes[i]))
                  for i in range(N))
    assert _chi2_ok(obs, exact, total, N)


def test_sampler_index_stream(oracle):
    g = synth.erdos_renyi(40, 5.0, seed=1)
    colors = synth.random_colors(g.n, 4, seed=1)
    T = oracle.Tables(g, colors, 4, 64)
    a = T.sample(4, seed=7, first_index=0, count=50)
    b = T.sample(4, seed=7, first_index=20, count=10)
    for x, y in zip(a, b):
        assert (x[20:30] == y).all()
    c = T.sample(4, seed=8, first_index=0, count=50)
    assert not (a[0] == c[0]).all()


def test_samples_are_colourful_connected_and_classified(oracle):
    k = 5
    g = synth.chung_lu(300, 1500, 2.5, seed=3)
    colors = synth.random_colors(g.n, k, seed=3)
    T = oracle.Tables(g, colors, k, 64)
    nodes, roots, shapes, classes = T.sample(k, seed=1, first_index=0, count=500)
    adj = brute.adjacency(g)
    for i in range(500):
        S = [int(x) for x in nodes[i]]
        assert S == sorted(set(S)) and len(S) == k
        assert len({int(colors[v]) for v in S}) == k
        assert int(roots[i]) in S
        assert brute.is_connected(adj, S)
        assert classes[i] == oracle.class_of_word(k, brute.word_of(adj, S))


def test_uniform_estimator_is_unbiased(oracle):
    k = 4
    g = synth.erdos_renyi(14, 5.0, seed=6)
    colors = synth.balanced_colors(g.n, k, seed=6)
    T = oracle.Tables(g, colors, k, 64)
    truth = brute.colourful_graphlets(g, colors, k, lambda w: oracle.class_of_word(k, w))
    s_i, _ = oracle.sigma(k)
    t = T.total(k)[1]
    N = 200_000
    est, hits = T.estimate_uniform(k, seed=3, n_samples=N)
    assert int(hits.sum()) == N
    p = 1.0 / oracle.inv_colorful_prob(k, k)
    for i in range(len(s_i)):
        c = truth.get(i, 0)
        q = c * int(s_i[i]) / t
        sd = t / int(s_i[i]) * math.sqrt(q * (1 - q) / N)
        assert abs(est[i] * p - c) <= 5 * sd + 1e-9, (i, est[i] * p, c)
    # the hits are exactly the classes of the same sample stream
    _, _, _, cls = T.sample(k, seed=3, first_index=0, count=N)
    assert (np.bincount(cls, minlength=len(s_i)) == hits).all()


def test_ags_multiplicative_guarantee(oracle):
    # Theorem 3: with probability 1 - delta every estimate is within 1 +- eps
    k = 4
    g = synth.erdos_renyi(16, 6.0, seed=2)
    colors = synth.balanced_colors(g.n, k, seed=2)
    T = oracle.Tables(g, colors, k, 64)
    truth = brute.colourful_graphlets(g, colors, k, lambda w: oracle.class_of_word(k, w))
    s = oracle.num_classes(k)
    assert len(truth) == s  # every 4-graphlet occurs colourfully
    eps, delta = 0.25, 0.1
    cbar = oracle.ags_cbar(eps, delta, s)
    est, hits, stats = T.estimate_ags(k, seed=5, max_samples=2_000_000, cbar=cbar)
    assert stats["covered"] == s and stats["switches"] == s
    p = 1.0 / oracle.inv_colorful_prob(k, k)
    for i in range(s):
        assert abs(est[i] * p - truth[i]) <= eps * truth[i], (i, est[i] * p, truth[i])


def test_ags_finds_graphlets_uniform_misses(oracle):
    # a hub with many leaves beside a small dense component: nearly every
    # colourful 4-treelet is a star at the hub, so uniform sampling spends
    # its budget there, while AGS covers the star graphlet, switches to the
    # path treelet (which the hub cannot span) and covers the rest
    # (Section 4.1)
    k = 4
    hub = synth.star(2000)
    corner = synth.erdos_renyi(20, 7.0, seed=3)
    n = hub.n + corner.n
    src = np.concatenate([np.repeat(np.arange(hub.n), hub.degrees()),
                          hub.n + np.repeat(np.arange(corner.n), corner.degrees())])
    dst = np.concatenate([hub.col.astype(np.int64), hub.n + corner.col.astype(np.int64)])
    g = synth.from_edges(n, src, dst)
    colors = synth.balanced_colors(n, k, seed=1)
    T = oracle.Tables(g, colors, k, 64)
    budget = 20_000
    _, hits_u = T.estimate_uniform(k, seed=2, n_samples=budget)
    _, hits_a, stats = T.estimate_ags(k, seed=2, max_samples=budget, cbar=200)
    assert (hits_u > 0).sum() <= 2
    assert stats["covered"] == oracle.num_classes(k) and stats["samples"] < budget
