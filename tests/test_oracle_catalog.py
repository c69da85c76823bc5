"""Pins for the oracle's treelet catalogue (Section 3.2.1, Section 3.3.1)."""
import math

from oracle import catalog as cat

# OEIS A000081 (rooted trees) and A000055 (unrooted trees), n = 1..8
ROOTED = [1, 1, 2, 4, 9, 20, 48, 115]
UNROOTED = [1, 1, 1, 2, 3, 6, 11, 23]


def test_rooted_and_unrooted_counts():
    assert [len(cat.rooted_shapes(h)) for h in range(1, 9)] == ROOTED
    assert [len(cat.unrooted_shapes(h)) for h in range(1, 9)] == UNROOTED


def test_1991_coloured_rooted_treelets():
    # Section 3.3.1: exactly 1991 rooted coloured treelets on at most 8 nodes
    assert sum(len(cat.rooted_shapes(h)) * math.comb(8, h) for h in range(1, 9)) == 1991


def test_figure1_encoding():
    # Figure 1: root coloured 3 with children 1 (children 2 and 7) and 5.
    adj = {3: [1, 5], 1: [3, 2, 7], 2: [1], 7: [1], 5: [3]}
    assert cat.encode(adj, 3) == "11010010"
    # s_C: bit l set for colour l, drawn most significant bit first
    mask = sum(1 << c for c in (3, 1, 2, 7, 5))
    assert format(mask, "08b") == "10101110"


def test_labelled_tree_counts_pin_automorphisms():
    # Cayley: h^(h-1) labelled rooted trees, h^(h-2) labelled trees
    for h in range(1, 9):
        f = math.factorial(h)
        rooted = sum(f // cat.root_automorphisms(s) for s in cat.rooted_shapes(h))
        assert rooted == h ** (h - 1)
        seen = {}
        for s in cat.rooted_shapes(h):
            seen.setdefault(cat.unrooted_code(s), s)
        unrooted = sum(f // cat.tree_automorphisms(s) for s in seen.values())
        assert unrooted == (h ** (h - 2) if h >= 2 else 1)


def test_decomposition_merges_back():
    # merging T' and T'' (1, s_T'', 0, s_T') gives T; T'' is the largest child
    for h in range(2, 9):
        for s in cat.rooted_shapes(h):
            a, b, beta = cat.decompose(s)
            assert "1" + b + "0" + a == s
            kids = cat._split_children(s)
            assert all(c <= kids[0] for c in kids)  # lexicographic on strings
            assert beta == kids.count("1" + b + "0") >= 1
            assert len(a) // 2 + 1 + len(b) // 2 + 1 == h


def test_shape_ids_ascend_with_encoding():
    for h in range(2, 9):
        vals = [int(s, 2) for s in cat.rooted_shapes(h)]
        assert vals == sorted(vals) and len(set(vals)) == len(vals)
        assert all(len(s) == 2 * (h - 1) for s in cat.rooted_shapes(h))


def test_catalog_flattening():
    c = cat.Catalog(8)
    assert len(c.strings) == sum(ROOTED)
    for g, s in enumerate(c.strings):
        if c.size[g] > 1:
            a, b = c.left[g], c.right[g]
            assert c.size[a] + c.size[b] == c.size[g]
            assert "1" + c.strings[b] + "0" + c.strings[a] == s
