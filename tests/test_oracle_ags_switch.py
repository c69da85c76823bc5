"""Pin of AGS's treelet-switch rule in the oracle (Algorithm AGS, Section 4.1).

When a graphlet becomes covered, AGS moves to the treelet T_j minimising
(1/t_j) * sum over covered graphlets i of sigma_ij * c_i / w_i, with
w_i = sum_j n_j sigma_ij / t_j.  Here the test replays the whole run itself
in exact rational arithmetic from values it finds by brute force:

* sigma_ij: the spanning trees of each graphlet class graph, listed edge
  subset by edge subset and sorted by tree shape;
* t_j: sum_i g_i sigma_ij with g_i the colourful induced copies of class i,
  found by listing node subsets (and checked against the oracle's totals);
* the samples: drawn from the oracle's sampler, whose exact distribution is
  pinned elsewhere, with the index streams of the algorithm (the n-th sample
  drawn with T_j has index first_index + j * 2^40 + n).

The oracle's first treelet, the treelet chosen at every switch, the number
of samples drawn by then and the weights w_i it used must equal the replay's.
Each case is chosen so that three plausible mistakes in the rule -- dropping
the 1/t_j factor, summing over the uncovered graphlets instead of the
covered ones, breaking ties towards the larger j -- pick another treelet at
some switch, so none of them could pass.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import brute


def _sigma_brute(oracle, h):
    """[class][unrooted shape] spanning trees, by enumeration."""
    shapes = cat.unrooted_shapes(h)
    out = []
    for w in oracle.class_codes(h):
        adj = brute.graph_of_word(h, int(w))
        row = [0] * len(shapes)
        for tree in brute.spanning_trees(adj, list(range(h))):
            ta = {v: [] for v in range(h)}
            for a, b in tree:
                ta[a].append(b)
                ta[b].append(a)
            row[shapes.index(min(int(cat.encode(ta, r), 2) for r in range(h)))] += 1
        out.append(row)
    return out


def _replay(T, h, sig, t, seed, cbar, max_samples, batch=4096):
    """Algorithm AGS in exact arithmetic; returns the first treelet, per
    switch (samples drawn, treelet chosen, weights, would each mutant rule
    choose differently), hits and the final weights."""
    nu, ncls = len(t), len(sig)
    live = [j for j in range(nu) if t[j] > 0]
    cur = min(live, key=lambda j: (-t[j], j))          # most frequent, ties to the smaller j
    first = cur
    hits, n = [0] * ncls, [0] * nu
    covered: list[int] = []
    drawn, trace = 0, []

    def weights():
        return [sum((Fraction(n[j] * sig[i][j], t[j]) for j in live), Fraction(0)) for i in range(ncls)]

    while len(covered) < ncls and drawn < max_samples:
        b = min(batch, max_samples - drawn)
        cls = T.sample(h, seed, (cur << 40) + n[cur], b, unrooted=cur)[3]
        for q in range(b):
            i = int(cls[q])
            n[cur] += 1
            drawn += 1
            hits[i] += 1
            if hits[i] == cbar and i not in covered:
                covered.append(i)
                w = weights()

                def score(j, over_covered=True, with_inverse=True):
                    idx = [a for a in range(ncls) if (a in covered) == over_covered and w[a] > 0]
                    acc = sum((Fraction(sig[a][j] * hits[a]) / w[a] for a in idx), Fraction(0))
                    return acc / t[j] if with_inverse else acc

                val = {j: score(j) for j in live}
                cur = min(live, key=lambda j: (val[j], j))
                mutants = (
                    min(live, key=lambda j: (score(j, with_inverse=False), j)) != cur,
                    min(live, key=lambda j: (score(j, over_covered=False), j)) != cur,
                    min(live, key=lambda j: (val[j], -j)) != cur,
                )
                trace.append((drawn, cur, w, mutants))
                break
    return first, trace, hits, weights()


CASES = [
    # (k, n, average degree, graph seed, cbar)
    (5, 16, 4.0, 0, 20),
    (6, 16, 4.0, 1, 20),
]


@pytest.mark.parametrize("k,n,deg,gseed,cbar", CASES)
def test_ags_switch_sequence_equals_exact_replay(oracle, k, n, deg, gseed, cbar):
    g = synth.erdos_renyi(n, deg, seed=gseed)
    colors = synth.balanced_colors(g.n, k, seed=gseed)
    T = oracle.Tables(g, colors, k, 64)
    sig = _sigma_brute(oracle, k)
    nu, ncls = len(cat.unrooted_shapes(k)), len(sig)
    # t_j from brute-force colourful graphlet counts, checked against the oracle
    gcount = brute.colourful_graphlets(g, colors, k, lambda w: oracle.class_of_word(k, w))
    t = [sum(gcount.get(i, 0) * sig[i][j] for i in range(ncls)) for j in range(nu)]
    assert t == [T.total(k, j)[1] for j in range(nu)]
    assert all(x > 0 for x in t)

    seed, max_samples = 3, 100_000
    first, trace, hits, w_end = _replay(T, k, sig, t, seed, cbar, max_samples)
    est, ohits, st = T.estimate_ags(k, seed=seed, max_samples=max_samples, cbar=cbar, trace=True)

    assert st["first"] == first
    assert st["switches"] == len(trace) and st["covered"] == len(trace)
    assert list(st["trace_j"]) == [tr[1] for tr in trace]
    assert list(st["trace_at"]) == [tr[0] for tr in trace]
    for s, (_, _, w, _) in enumerate(trace):
        exact = np.array([float(x) for x in w])
        assert np.allclose(st["trace_w"][s], exact, rtol=1e-13, atol=0), s
    assert [int(x) for x in ohits] == hits
    ip = oracle.inv_colorful_prob(k, k)
    want = np.array([float(Fraction(hits[i]) / w_end[i]) * ip if w_end[i] > 0 else 0.0
                     for i in range(ncls)])
    assert np.allclose(est, want, rtol=1e-12, atol=0)

    # the case tells each plausible mistake apart from the rule
    mut = np.array([tr[3] for tr in trace])
    assert mut[:, 0].any(), "dropping 1/t_j would choose the same treelets"
    assert mut[:, 1].any(), "summing over uncovered graphlets would choose the same treelets"
    assert mut[:, 2].any(), "ties towards the larger j would choose the same treelets"


def test_ags_sample_budget_fits_the_index_streams(oracle):
    # each treelet's stream holds 2^40 indices, so a larger budget is refused
    g = synth.erdos_renyi(16, 4.0, seed=0)
    colors = synth.balanced_colors(g.n, 4, seed=0)
    T = oracle.Tables(g, colors, 4, 64)
    with pytest.raises(Exception):
        T.estimate_ags(4, seed=1, max_samples=(1 << 40) + 1, cbar=20)
    T.estimate_ags(4, seed=1, max_samples=1000, cbar=20)
