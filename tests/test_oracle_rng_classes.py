"""Pins for the oracle's random numbers, colouring, graphlet classes and
spanning-tree counts (Section 2.1, Section 4.4.3)."""
import itertools
import math
import random

import numpy as np
import pytest

from oracle import catalog as cat
from tests import brute


def test_philox_known_answers(oracle):
    # Known-answer vectors published with the Random123 library for
    # philox4x32 with 10 rounds (counter, key -> output)
    kat = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in kat:
        assert oracle.philox4x32_10(ctr, key) == want


def test_colouring_uses_first_word(oracle):
    seed, k = 0x1234_5678_9ABC, 7
    cols = oracle.color(100, k, seed)
    for v in range(100):
        x0 = oracle.philox4x32_10((v, 0, 0, 0xC010), (seed & 0xFFFFFFFF, seed >> 32))[0]
        assert cols[v] == (x0 * k) >> 32


def test_colouring_is_uniform(oracle):
    k, n = 5, 200_000
    cols = oracle.color(n, k, 3)
    counts = np.bincount(cols, minlength=k)
    chi2 = float(((counts - n / k) ** 2 / (n / k)).sum())
    assert chi2 < 20.5  # 4 d.o.f., p ~ 4e-4


def test_draw_below_contract(oracle):
    seed = 99
    for W in (1, 2, 3, 5, 1000, 2**63 + 5, 2**64 + 1, 2**127 + 3, 2**128 - 1):
        for idx in range(20):
            r = oracle.draw_below(seed, idx, 3, W)
            assert 0 <= r < W
            # first accepted attempt of the masked 128-bit word
            b = (W - 1).bit_length()
            for att in range(64):
                x = oracle.philox4x32_10((idx, 0, 3, att), (seed, 0))
                word = x[0] | x[1] << 32 | x[2] << 64 | x[3] << 96
                word &= (1 << b) - 1
                if word < W:
                    assert r == word
                    break


def test_draw_below_uniform(oracle):
    W, N = 6, 60_000
    counts = np.bincount([oracle.draw_below(5, i, 1, W) for i in range(N)], minlength=W)
    chi2 = float(((counts - N / W) ** 2 / (N / W)).sum())
    assert chi2 < 25.7  # 5 d.o.f.


# OEIS A001349: connected graphs on n nodes; the paper quotes N_8 = 11117
CONNECTED = [1, 1, 2, 6, 21, 112, 853]


def test_class_counts(oracle):
    assert [oracle.num_classes(h) for h in range(1, 8)] == CONNECTED


@pytest.mark.slow
def test_class_count_k8(oracle):
    assert oracle.num_classes(8) == 11117


def test_class_codes_are_orbit_minima(oracle):
    for h in range(2, 7):
        codes = oracle.class_codes(h)
        assert (np.diff(codes.astype(np.int64)) > 0).all()
        for w in codes[:: max(1, len(codes) // 40)]:
            assert oracle.canonical_code(h, int(w)) == int(w)
            assert brute.is_connected(brute.graph_of_word(h, int(w)), range(h))


def test_canonical_code_is_relabelling_invariant(oracle):
    rng = random.Random(3)
    for h in (4, 5, 6, 7):
        for _ in range(30):
            adj = [set() for _ in range(h)]
            for i, j in itertools.combinations(range(h), 2):
                if rng.random() < 0.5:
                    adj[i].add(j)
                    adj[j].add(i)
            w = brute.word_of(adj, range(h))
            perm = list(range(h))
            rng.shuffle(perm)
            adj2 = [set() for _ in range(h)]
            for i in range(h):
                for j in adj[i]:
                    adj2[perm[i]].add(perm[j])
            w2 = brute.word_of(adj2, range(h))
            assert oracle.canonical_code(h, w) == oracle.canonical_code(h, w2)
            conn = brute.is_connected(adj, range(h))
            assert (oracle.class_of_word(h, w) >= 0) == conn


def test_word_bit_order(oracle):
    # the path 0-1-2-3: pairs (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) -> 100101
    adj = [{1}, {0, 2}, {1, 3}, {2}]
    assert brute.word_of(adj, range(4)) == 0b100101


def _word(h, edges):
    adj = [set() for _ in range(h)]
    for a, b in edges:
        adj[a].add(b)
        adj[b].add(a)
    return brute.word_of(adj, range(h))


def test_kirchhoff_closed_forms(oracle):
    for h in range(2, 9):
        K = _word(h, itertools.combinations(range(h), 2))
        assert oracle.spanning_trees(h, K) == h ** (h - 2)          # Cayley
        P = _word(h, [(i, i + 1) for i in range(h - 1)])
        assert oracle.spanning_trees(h, P) == 1
        if h >= 3:
            Cy = _word(h, [(i, (i + 1) % h) for i in range(h)])
            assert oracle.spanning_trees(h, Cy) == h


def test_sigma_k4_table(oracle):
    s_i, s_ij = oracle.sigma(4)
    # unrooted 4-shapes: star (id 0), path (id 1)
    got = {}
    for c, w in enumerate(oracle.class_codes(4)):
        adj = brute.graph_of_word(4, int(w))
        m = sum(len(a) for a in adj) // 2
        got[m, max(len(a) for a in adj)] = (int(s_i[c]), tuple(int(x) for x in s_ij[c]))
    assert got == {(3, 2): (1, (0, 1)),      # path
                   (3, 3): (1, (1, 0)),      # star
                   (4, 2): (4, (0, 4)),      # C4
                   (4, 3): (3, (1, 2)),      # paw
                   (5, 3): (8, (2, 6)),      # diamond
                   (6, 3): (16, (4, 12))}    # K4


@pytest.mark.parametrize("h", [3, 4, 5])
def test_sigma_ij_brute_force(oracle, h):
    s_i, s_ij = oracle.sigma(h)
    shapes = cat.unrooted_shapes(h)
    for c, w in enumerate(oracle.class_codes(h)):
        adj = brute.graph_of_word(h, int(w))
        counts = [0] * len(shapes)
        for tree in brute.spanning_trees(adj, tuple(range(h))):
            ta = {v: [] for v in range(h)}
            for a, b in tree:
                ta[a].append(b)
                ta[b].append(a)
            counts[shapes.index(min(int(cat.encode(ta, r), 2) for r in range(h)))] += 1
        assert counts == [int(x) for x in s_ij[c]]
        assert sum(counts) == s_i[c]


@pytest.mark.parametrize("h", [6, 7])
def test_sigma_rows_sum_to_kirchhoff(oracle, h):
    s_i, s_ij = oracle.sigma(h)
    assert (s_ij.sum(axis=1) == s_i).all()
    # the clique's row: spanning trees of K_h of shape j are its h!/|Aut(T_j)| labellings
    K = oracle.class_codes(h)[-1]
    assert K == (1 << math.comb(h, 2)) - 1
    seen = {}
    for s in cat.rooted_shapes(h):
        seen.setdefault(cat.unrooted_code(s), s)
    want = [math.factorial(h) // cat.tree_automorphisms(seen[c]) for c in cat.unrooted_shapes(h)]
    assert [int(x) for x in s_ij[-1]] == want
