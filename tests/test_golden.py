"""The oracle against the values the paper prints (tests/golden/)."""
import math
import os

import synth
from oracle import catalog as cat

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden() -> dict:
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_values.txt")):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = (x.strip() for x in line.split("=", 1))
            out[k] = v
    return out


def test_figure1_encoding():
    g = _golden()
    adj = {}
    for e in g["figure1_edges"].split():
        a, b = (int(x) for x in e.split("-"))
        adj.setdefault(a, []).append(b)
        adj.setdefault(b, []).append(a)
    assert cat.encode(adj, int(g["figure1_root"])) == g["figure1_s_T"]
    colours = sorted(adj)
    s_c = "".join("1" if c in colours else "0" for c in range(7, -1, -1))
    assert s_c == g["figure1_s_C"]


def test_coloured_rooted_treelets_k8():
    k = 8
    total = sum(len(cat.rooted_shapes(h)) * math.comb(k, h) for h in range(1, k + 1))
    assert total == int(_golden()["coloured_rooted_treelets_k8"])


def test_graphlets_8(oracle):
    assert oracle.num_classes(8) == int(_golden()["graphlets_8"])


def test_k6_star_footnote(oracle):
    # the stars of a 2^16-leaf star graph, by the oracle's star index
    g = synth.star(1 << 16)
    T = oracle.Tables(g, oracle.color(g.n, 6, 0), 6, 128, nthreads=4)
    want = float(_golden()["stars_k6_degree_2_16_approx"])
    got = T.star_total(6)
    assert got == math.comb(1 << 16, 5)
    assert abs(got / want - 1) < 0.05   # "about 10^22"
