"""R-MAT graphs (a, b, c = 0.57, 0.19, 0.19) with k = 7 and 128-bit counts.

Scale 13 (8k nodes, edge factor 16): every table entry, total, sample and
class, the uniform and the adaptive estimates against the oracle.

Scale 22 (4.2M nodes, 64M edges, maximum degree ~160k): closed forms that
hold at any size, and sampled outputs checked one by one.  The colourful
h-star has a unique centre for h >= 3, and its copies centred at v are the
choices of h - 1 neighbours of distinct colours other than c_v: the total of
the star shape is the sum over v of the elementary symmetric polynomial
e_{h-1} of v's per-colour neighbour counts.  An edge is colourful when its
ends differ in colour, so the level-2 total is the number of bichromatic
edges.  2000 samples of each size 5..7 must be colourful, connected, and
carry the oracle's canonical class of their induced adjacency word.  10M
adaptive samples (Section 4.1) must account for every hit.
"""
import os

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import brute, layout

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

K, BITS = 7, 128


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    return M


def _ulp_close(a, b, ulps=2):
    ia = np.asarray(a, np.float64).view(np.int64)
    ib = np.asarray(b, np.float64).view(np.int64)
    return bool(np.all(np.abs(ia - ib) <= ulps))


def test_rmat13_k7_against_oracle(M, oracle):
    g = synth.rmat(13, 16, seed=1)
    G = M.Graph.from_csr(g)
    gcol = M.color(G, K, 77)
    colors = gcol.cpu().numpy()
    T = M.Tables(G, gcol, K, BITS)
    O = oracle.Tables(g, colors, K, BITS, nthreads=os.cpu_count())
    C = cat.Catalog(K)
    for h in range(1, K + 1):
        assert np.array_equal(layout.gpu_c_as_oracle(T.read(h, 0), colors, K, h, C.r(h)),
                              O.level(h)), h
        assert T.total(h) == O.total(h)
        for j in range(len(cat.unrooted_shapes(h))):
            assert T.total(h, j) == O.total(h, j)
    for h, seed in ((7, 3), (6, 4), (5, 5)):
        gn, gr, gsh, gcl = T.sample(h, seed, 0, 3000)
        on, orr, osh, ocl = O.sample(h, seed, 0, 3000)
        assert np.array_equal(gn.cpu().numpy().astype(np.uint32), on)
        assert np.array_equal(gr.cpu().numpy().astype(np.uint32), orr)
        assert np.array_equal(gsh.cpu().numpy(), osh)
        assert np.array_equal(gcl.cpu().numpy(), ocl)
    est, hits, _ = T.estimate(K, seed=6, samples=50_000)
    oest, ohits = O.estimate_uniform(K, seed=6, n_samples=50_000)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
    est, hits, st = T.estimate(K, seed=8, samples=300_000, mode=M.MC_EST_AGS, cbar=100)
    oest, ohits, ost = O.estimate_ags(K, seed=8, max_samples=300_000, cbar=100)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
    assert (st["samples"], st["switches"], st["covered"]) == \
        (ost["samples"], ost["switches"], ost["covered"])


def _has_edge(g, a, b) -> bool:
    row = g.col[g.row_ptr[a]:g.row_ptr[a + 1]]
    i = np.searchsorted(row, b)
    return bool(i < len(row) and row[i] == b)


def test_rmat22_k7_full_size(M, oracle):
    g = synth.rmat(22, 16, seed=0)
    G = M.Graph.from_csr(g, trusted=True)
    gcol = M.color(G, K, 2022)
    colors = gcol.cpu().numpy()
    T = M.Tables(G, gcol, K, BITS)
    stars = brute.star_totals(g, colors, K)
    assert T.total(2) == (2 * stars[2], stars[2])
    for h in range(3, K + 1):
        j = cat.unrooted_id("10" * (h - 1))
        assert T.total(h, j)[1] == stars[h], h
        R, U = T.total(h)
        assert R == h * U
        assert sum(T.total(h, jj)[1] for jj in range(len(cat.unrooted_shapes(h)))) == U
    for h in (5, 6, 7):
        nodes, _, _, cls = T.sample(h, 11 + h, 0, 2000, roots=False, shapes=False)
        nodes = nodes.cpu().numpy().astype(np.int64)
        cls = cls.cpu().numpy()
        for s in range(2000):
            vs = nodes[s]
            assert np.all(np.diff(vs) > 0)
            assert len(set(colors[vs].tolist())) == h
            w = 0
            adj = {i: [] for i in range(h)}
            for a in range(h):
                for b in range(a + 1, h):
                    e = _has_edge(g, vs[a], vs[b])
                    w = (w << 1) | int(e)
                    if e:
                        adj[a].append(b)
                        adj[b].append(a)
            seen, stack = {0}, [0]
            while stack:
                x = stack.pop()
                for y in adj[x]:
                    if y not in seen:
                        seen.add(y)
                        stack.append(y)
            assert len(seen) == h
            assert cls[s] == oracle.class_of_word(h, w)
    est, hits, st = T.estimate(K, seed=5, samples=10_000_000, mode=M.MC_EST_AGS, cbar=1000)
    assert int(hits.sum()) == st["samples"] <= 10_000_000
    assert np.all(np.isfinite(est)) and np.all(est >= 0)
    assert np.all((est > 0) == (hits > 0))
