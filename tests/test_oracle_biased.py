"""Pins for biased colouring (Section 3.5) in the oracle.

* Colour frequencies follow (1 - (k-1) lambda, lambda, ..., lambda) (chi-square);
  lambda = 0 is the uniform colouring.
* 1/p: p summed over all colour assignments of h nodes with distinct
  colours, in exact rationals.
* Over all k^n colourings of a small graph, weighted by their
  probabilities, the expected colourful copies of every tree and every
  graphlet are exactly p times their number -- so dividing colourful
  estimates by this p is unbiased.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import brute

LAM = [3 * 2**28, 2**29 + 12345, 12_345_678]  # lambda = 0.1875, ~0.125, ~0.0029


@pytest.mark.parametrize("k,L", [(4, LAM[0]), (5, LAM[1]), (8, LAM[2])])
def test_biased_colour_frequencies(oracle, k, L):
    n = 400_000
    c = oracle.color_biased(n, k, 7, L)
    lam = L / 2**32
    want = np.array([1 - (k - 1) * lam] + [lam] * (k - 1)) * n
    got = np.bincount(c, minlength=k)
    chi2 = float(((got - want) ** 2 / want).sum())
    assert chi2 < (k - 1) + 6 * math.sqrt(2 * (k - 1))
    assert np.array_equal(oracle.color_biased(1000, k, 3, 0), oracle.color(1000, k, 3))
    with pytest.raises(oracle.OracleError):
        oracle.color_biased(10, k, 1, 2**32 // (k - 1) + 1)


def _p_exact(k, h, L):
    lam = Fraction(L, 2**32)
    probs = [1 - (k - 1) * lam] + [lam] * (k - 1)
    tot = Fraction(0)
    for cols in itertools.product(range(k), repeat=h):
        if len(set(cols)) == h:
            w = Fraction(1)
            for c in cols:
                w *= probs[c]
            tot += w
    return tot


@pytest.mark.parametrize("k", [3, 4, 5, 6, 7])
def test_biased_colourful_probability(oracle, k):
    for L in LAM + [0]:
        if (k - 1) * L > 2**32:
            continue
        for h in range(2, k + 1):
            p = _p_exact(k, h, L) if L else Fraction(math.factorial(k), math.factorial(k - h) * k**h)
            got = oracle.inv_colorful_prob_biased(k, h, L)
            assert abs(got * p - 1) < 1e-14, (k, h, L)


def test_biased_expectation_over_all_colourings(oracle):
    k, L = 4, LAM[0]
    lam = Fraction(L, 2**32)
    probs = [1 - (k - 1) * lam] + [lam] * (k - 1)
    g = synth.erdos_renyi(6, 3.0, seed=2)
    copies = brute.tree_copies(g, k)
    classify = lambda w: oracle.class_of_word(k, w)
    truth = brute.graphlets(g, k, classify)
    shapes = cat.unrooted_shapes(k)
    acc_t = [Fraction(0)] * len(shapes)
    acc_g = {}
    for cols in itertools.product(range(k), repeat=g.n):
        w = Fraction(1)
        for c in cols:
            w *= probs[c]
        colors = np.array(cols, np.uint8)
        T = oracle.Tables(g, colors, k, 64, nthreads=1)
        for j in range(len(shapes)):
            acc_t[j] += w * T.total(k, j)[1]
        for i, c in brute.colourful_graphlets(g, colors, k, classify).items():
            acc_g[i] = acc_g.get(i, 0) + w * c
    p = 1 / Fraction(oracle.inv_colorful_prob_biased(k, k, L))
    pe = _p_exact(k, k, L)
    assert abs(p / pe - 1) < 1e-14
    for j, code in enumerate(shapes):
        assert acc_t[j] == pe * copies.get(code, 0)
    for i, gi in truth.items():
        assert acc_g.get(i, 0) == pe * gi
