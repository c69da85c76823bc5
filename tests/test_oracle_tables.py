"""Pins for the oracle's count tables c(T_C, v) (Section 2.1, Eq. 1).

Brute-force enumeration of colourful treelet copies on tiny graphs, closed
forms on cliques, stars and paths, the colouring-average invariant
(E[colourful copies] = p_k * copies, Section 2.2) and overflow behaviour.
"""
import itertools
import math

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import brute


def _table_dict(T, h):
    """{(v, s_T, mask): count} of the non-zero entries of level h."""
    lv = T.level_int(h)
    masks = [m for m in range(1 << T.k) if bin(m).count("1") == h]
    out = {}
    for v in range(T.n):
        for s_i, s in enumerate(cat.rooted_shapes(h)):
            for q, m in enumerate(masks):
                if lv[v][s_i][q]:
                    out[(v, s, m)] = lv[v][s_i][q]
    return out


def _tiny_graphs():
    yield synth.erdos_renyi(9, 3.5, seed=1)
    yield synth.erdos_renyi(10, 4.0, seed=2)
    yield synth.clique(6)
    yield synth.cycle(7)
    yield synth.star(6)
    yield synth.lollipop(5, 3)
    yield synth.grid_road(3, seed=0, p_diag=0.5)


@pytest.mark.parametrize("k", [3, 4, 5])
def test_tables_match_brute_force(oracle, k):
    for gi, g in enumerate(_tiny_graphs()):
        colors = synth.random_colors(g.n, k, seed=10 + gi)
        T = oracle.Tables(g, colors, k, 128, nthreads=2)
        for h in range(1, k + 1):
            assert _table_dict(T, h) == brute.treelet_counts(g, colors, h), (g.name, k, h)


def test_tables_k6_brute_force(oracle):
    g = synth.erdos_renyi(9, 4.5, seed=5)
    colors = synth.random_colors(g.n, 6, seed=3)
    T = oracle.Tables(g, colors, 6, 128, nthreads=2)
    for h in (5, 6):
        assert _table_dict(T, h) == brute.treelet_counts(g, colors, h)


def test_clique_closed_form(oracle):
    # K_n: c(T_C, v) = prod_{a in C \ {c_v}} n_a * (h-1)! / |Aut_root(T)|
    k, g = 5, synth.clique(11)
    colors = synth.random_colors(g.n, k, seed=7)
    na = np.bincount(colors, minlength=k)
    T = oracle.Tables(g, colors, k, 128)
    for h in range(1, k + 1):
        lv = T.level_int(h)
        masks = [m for m in range(1 << k) if bin(m).count("1") == h]
        for v in range(g.n):
            cv = int(colors[v])
            for s_i, s in enumerate(cat.rooted_shapes(h)):
                for q, m in enumerate(masks):
                    if not m >> cv & 1:
                        want = 0
                    else:
                        want = math.factorial(h - 1) // cat.root_automorphisms(s)
                        for a in range(k):
                            if a != cv and m >> a & 1:
                                want *= int(na[a])
                    assert lv[v][s_i][q] == want


def test_star_closed_form(oracle):
    # star centred at 0: c(star rooted at centre, C, 0) = prod_{a in C \ {c_0}} n_a
    k, g = 5, synth.star(40)
    colors = synth.random_colors(g.n, k, seed=1)
    na = np.bincount(colors[1:], minlength=k)
    T = oracle.Tables(g, colors, k, 128)
    c0 = int(colors[0])
    for h in range(2, k + 1):
        star_s = "10" * (h - 1)
        s_i = cat.rooted_shapes(h).index(star_s)
        masks = [m for m in range(1 << k) if bin(m).count("1") == h]
        lv = T.level_int(h)
        for q, m in enumerate(masks):
            want = 0
            if m >> c0 & 1:
                want = 1
                for a in range(k):
                    if a != c0 and m >> a & 1:
                        want *= int(na[a])
            assert lv[0][s_i][q] == want
            for other in range(len(cat.rooted_shapes(h))):
                if other != s_i:
                    assert lv[0][other][q] == 0


def test_path_closed_form(oracle):
    # P_n: colourful k-paths = windows of k consecutive nodes with distinct colours
    k, g = 5, synth.path(60)
    colors = synth.random_colors(g.n, k, seed=4)
    T = oracle.Tables(g, colors, k, 128)
    windows = sum(1 for i in range(g.n - k + 1) if len(set(colors[i:i + k].tolist())) == k)
    path_code = min(int(cat.encode(cat.decode("1" * (k - 1) + "0" * (k - 1)), r), 2)
                    for r in range(k))
    j = cat.unrooted_shapes(k).index(path_code)
    assert T.total(k, j)[1] == windows
    assert T.total(k)[1] == windows


def test_colouring_average_invariant(oracle):
    # Over all k^n colourings, sum of colourful copies of each tree shape j
    # = k! k^(n-k) * (number of copies of j): each k-node copy is colourful
    # under k! k^(n-k) colourings.
    k = 4
    g = synth.erdos_renyi(7, 3.0, seed=3)
    copies = brute.tree_copies(g, k)
    shapes = cat.unrooted_shapes(k)
    acc = [0] * len(shapes)
    for colors in itertools.product(range(k), repeat=g.n):
        T = oracle.Tables(g, np.array(colors, np.uint8), k, 64, nthreads=1)
        for j in range(len(shapes)):
            acc[j] += T.total(k, j)[1]
    for j, code in enumerate(shapes):
        assert acc[j] == math.factorial(k) * k ** (g.n - k) * copies.get(code, 0)


def test_totals_are_rooted_over_h(oracle):
    g = synth.erdos_renyi(60, 6.0, seed=9)
    colors = synth.random_colors(g.n, 5, seed=2)
    T = oracle.Tables(g, colors, 5, 64)
    for h in range(2, 6):
        R, U = T.total(h)
        assert R == h * U
        parts = [T.total(h, j) for j in range(len(cat.unrooted_shapes(h)))]
        assert sum(p[0] for p in parts) == R
        assert sum(p[1] for p in parts) == U


def test_overflow_u64_vs_u128(oracle):
    # a star with 2^16 leaves and k = 6: prod over five colour classes of
    # ~2^16/6 leaves exceeds 2^64 (the paper's Section 3.2.1 example)
    k, g = 6, synth.star(1 << 16)
    colors = synth.random_colors(g.n, k, seed=0)
    with pytest.raises(oracle.OracleOverflow):
        oracle.Tables(g, colors, k, 64, nthreads=4)
    T = oracle.Tables(g, colors, k, 128, nthreads=4)
    c0 = int(colors[0])
    na = np.bincount(colors[1:], minlength=k)
    want = 1
    for a in range(k):
        if a != c0:
            want *= int(na[a])
    lv = T.level(k)
    s_i = cat.rooted_shapes(k).index("10" * (k - 1))
    got = int(lv[0, s_i, 0, 0]) | (int(lv[0, s_i, 0, 1]) << 64)
    assert got == want > 2 ** 64


def test_neighbor_sum_definition(oracle):
    g = synth.erdos_renyi(30, 5.0, seed=1)
    colors = synth.random_colors(g.n, 4, seed=1)
    T = oracle.Tables(g, colors, 4, 64)
    for h in (1, 2, 3):
        lv = T.level(h).astype(object)
        for v in (0, 7, 29):
            S = T.neighbor_sum(h, v)
            want = sum(lv[int(u), :, :, 0] for u in g.neighbors(v))
            assert (S[:, :, 0].astype(object) == want).all()


@pytest.mark.parametrize("k", [3, 4, 5, 6])
def test_zero_rooting_keeps_each_copy_once(oracle, k):
    # Section 3.4.1: level-k counts only at colour-0 nodes.  Every colourful
    # k-treelet has exactly one colour-0 node, so the zero-rooted level k holds
    # each copy once: its total is t (= rooted total / k of the full table).
    for gi, g in enumerate([synth.erdos_renyi(40, 5.0, seed=k), synth.chung_lu(300, 1500, 2.4, seed=k)]):
        colors = synth.random_colors(g.n, k, seed=gi)
        A = oracle.Tables(g, colors, k, 128)
        Z = oracle.Tables(g, colors, k, 128, zero_root=True)
        for j in range(len(cat.unrooted_shapes(k))):
            assert Z.total(k, j) == (A.total(k, j)[1], A.total(k, j)[1])
        la, lz = A.level(k), Z.level(k)
        zero = colors == 0
        assert np.array_equal(la[zero], lz[zero]) and not lz[~zero].any()
        for h in range(1, k):
            assert np.array_equal(A.level(h), Z.level(h))


def test_star_totals_closed_form_any_graph(oracle):
    # For h >= 3 an h-star has one centre; its colourful copies centred at v
    # choose h-1 neighbours of distinct colours, none c_v: the star total is
    # sum_v e_{h-1}(per-colour neighbour counts of v without c_v).
    k = 6
    g = synth.rmat(9, 12, seed=3)
    colors = synth.random_colors(g.n, k, seed=5)
    T = oracle.Tables(g, colors, k, 128)
    stars = brute.star_totals(g, colors, k)
    assert T.total(2)[1] == stars[2]
    for h in range(3, k + 1):
        assert T.total(h, cat.unrooted_id("10" * (h - 1)))[1] == stars[h]


@pytest.mark.parametrize("k", [7, 8])
def test_tables_k7_k8_brute_force(oracle, k):
    # the treelet sizes of the R-MAT (k = 7) and serving (k = 8) workloads
    g = synth.erdos_renyi(k + 2, 4.0, seed=k)
    colors = synth.balanced_colors(g.n, k, seed=k)
    T = oracle.Tables(g, colors, k, 128, nthreads=2)
    for h in (k - 1, k):
        assert _table_dict(T, h) == brute.treelet_counts(g, colors, h), h
