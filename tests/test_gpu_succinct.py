"""Succinct tables (Section 3.2.1: non-zero entries only, per node sorted by
key) and variable-length counts (Section 3.3.3: each row's counts in the
fewest bytes that hold its largest) against the oracle and the dense tables.

The packed levels, read back as dense rows, equal the oracle's tables entry
by entry; samples, classes, totals and estimates drawn from them equal those
of the dense tables bit for bit (the sampler finds each entry by binary
search of its row's keys instead of indexing a dense row).
"""
import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests.test_gpu_parity import _ulp_close, assert_tables_equal, assert_totals_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    return M


def _same_samples(A, B, h, seed, count, unrooted=-1):
    a = A.sample(h, seed, 0, count, unrooted=unrooted)
    b = B.sample(h, seed, 0, count, unrooted=unrooted)
    for x, y in zip(a, b):
        assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())


CASES = [
    # graph, k, bits, varlen, flags
    (lambda: synth.chung_lu_scaled(20000, seed=1), 5, 64, False, {}),
    (lambda: synth.chung_lu_scaled(20000, seed=2), 5, 64, True, {}),
    (lambda: synth.chung_lu(5000, 30000, 2.3, seed=2), 6, 128, True, {}),
    (lambda: synth.chung_lu(3000, 12000, 2.3, seed=11), 8, 128, True, {}),
    (lambda: synth.chung_lu_scaled(15000, seed=3), 5, 64, True, {"zero_root": True}),
    (lambda: synth.chung_lu(5000, 30000, 2.3, seed=4), 6, 128, False, {"skip_round": True}),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_packed_tables(M, oracle, case):
    make, k, bits, varlen, flags = CASES[case]
    g = make()
    colors = oracle.color(g.n, k, 50 + case)
    G = M.Graph.from_csr(g)
    D = M.Tables(G, colors, k, bits, **flags)
    P = M.Tables(G, colors, k, bits, succinct=True, varlen=varlen, **flags)
    skip = flags.get("skip_round", False)
    levels = [h for h in range(1, k + 1) if not (skip and h == k - 1)]
    for h in levels:
        assert np.array_equal(P.read(h, 0), D.read(h, 0)), f"c level {h}"
        assert P.nonzeros(h, 0) == D.nonzeros(h, 0)
        if h < k:
            assert np.array_equal(P.read(h, 1), D.read(h, 1)), f"S level {h}"
            assert P.nonzeros(h, 1) == D.nonzeros(h, 1)
        assert P.total(h) == D.total(h)
    if not skip:
        O = oracle.Tables(g, colors, k, bits, **flags)
        assert_tables_equal(M, P, O, g, colors, k)
        assert_totals_equal(P, O, k)
    for j in range(len(cat.unrooted_shapes(k))):
        assert P.total(k, j) == D.total(k, j)
    n_s = 2000 if k < 8 else 500
    _same_samples(P, D, k, 7, n_s)
    _same_samples(P, D, k - 2, 8, 500)
    for j in range(0, len(cat.unrooted_shapes(k)), 3):
        if D.total(k, j)[0] > 0:
            _same_samples(P, D, k, 9, 200, unrooted=j)
    kw = {"star_samples": 2000} if skip else {}
    e1, h1, _ = P.estimate(k, seed=3, samples=5000, **kw)
    e2, h2, _ = D.estimate(k, seed=3, samples=5000, **kw)
    assert np.array_equal(h1, h2) and _ulp_close(e1, e2)
    e1, h1, s1 = P.estimate(k, seed=4, samples=50_000, mode=M.MC_EST_AGS, cbar=50, **kw)
    e2, h2, s2 = D.estimate(k, seed=4, samples=50_000, mode=M.MC_EST_AGS, cbar=50, **kw)
    assert np.array_equal(h1, h2) and _ulp_close(e1, e2) and s1["switches"] == s2["switches"]
    dense, stored = P.table_bytes()
    assert dense == D.table_bytes()[0] == D.table_bytes()[1]
    if varlen:
        assert stored < dense
    with pytest.raises(M.MotifError):
        P.rebuild(M.color(G, k, 1))


def test_packed_degenerate_inputs(M, oracle):
    # no nodes; isolated nodes only (every level above 1 all zeros); a path
    # (no 4-star, so some rows are empty); zero samples
    G = M.Graph(np.zeros(1, np.int64), np.zeros(0, np.uint32))
    T = M.Tables(G, np.zeros(0, np.uint8), 4, 64, succinct=True, varlen=True)
    assert T.total(4) == (0, 0) and T.table_bytes()[1] == 0
    g = synth.from_edges(50, [], [])
    G = M.Graph.from_csr(g)
    T = M.Tables(G, oracle.color(50, 3, 0), 3, 64, succinct=True)
    assert T.total(3) == (0, 0) and T.total(1) == (50, 50)
    assert T.nonzeros(2) == 0 and T.nonzeros(1, 1) == 0
    assert not T.read(3, 0).any()
    with pytest.raises(M.MotifError):
        T.sample(3, 1, 0, 10)
    g = synth.path(40)
    colors = oracle.color(g.n, 4, 2)
    G = M.Graph.from_csr(g)
    P = M.Tables(G, colors, 4, 128, succinct=True, varlen=True)
    D = M.Tables(G, colors, 4, 128)
    for h in range(1, 5):
        assert np.array_equal(P.read(h, 0), D.read(h, 0))
    if D.total(4)[0] > 0:
        _same_samples(P, D, 4, 5, 300)
    P.sample(4, 1, 0, 0)
