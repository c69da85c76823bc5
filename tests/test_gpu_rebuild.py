"""In-place rebuilds (mc_rebuild_tables), eagerly and replayed from a
captured CUDA graph: after rebuilding for colouring B, tables, totals,
samples and estimates equal those of a fresh build for B (and the oracle's),
whatever colouring came before; a bad colouring is reported by the next
call, and a later good rebuild clears it."""
import numpy as np
import pytest

import synth
from oracle import catalog as cat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    return M


def _same(A, B, k):
    for h in range(1, k + 1):
        assert np.array_equal(A.read(h, 0), B.read(h, 0)), h
        assert A.total(h) == B.total(h)
        for j in range(len(cat.unrooted_shapes(h))):
            assert A.total(h, j) == B.total(h, j)
    for h in range(1, k):
        assert np.array_equal(A.read(h, 1), B.read(h, 1)), h
    for h in range(3, k + 1):  # a level-h root index made before the rebuild is redone
        if A.total(h)[0] == 0:
            continue
        a = A.sample(h, 7, 0, 2000)
        b = B.sample(h, 7, 0, 2000)
        for x, y in zip(a, b):
            assert np.array_equal(x.cpu().numpy(), y.cpu().numpy())
    ea, ha, _ = A.estimate(k, seed=3, samples=20000)
    eb, hb, _ = B.estimate(k, seed=3, samples=20000)
    assert np.array_equal(ha, hb) and np.array_equal(ea, eb)


@pytest.mark.parametrize("k,bits,skip", [(5, 64, False), (6, 128, False), (6, 128, True)])
def test_rebuild_equals_fresh_build(M, oracle, k, bits, skip):
    import torch
    g = synth.chung_lu_scaled(20000, seed=k)
    G = M.Graph.from_csr(g)
    ca = M.color(G, k, 1, out=torch.empty(g.n, dtype=torch.uint8, device="cuda"))
    cb = M.color(G, k, 2, out=torch.empty(g.n, dtype=torch.uint8, device="cuda"))
    T = M.Tables(G, ca, k, bits, skip_round=skip)
    levels = [h for h in range(2, k) if not (skip and h == k - 1)]
    for h in levels:
        T.total(h)  # root indices of lower levels, built for colouring A
    T.rebuild(cb)
    F = M.Tables(G, cb, k, bits, skip_round=skip)
    if skip:
        for h in levels + [k]:
            assert np.array_equal(T.read(h, 0), F.read(h, 0))
            assert T.total(h) == F.total(h)
        est, hits, _ = T.estimate(k, seed=3, samples=20000, star_samples=2000)
        oest, ohits, _ = F.estimate(k, seed=3, samples=20000, star_samples=2000)
        assert np.array_equal(hits, ohits) and np.array_equal(est, oest)
    else:
        _same(T, F, k)
        O = oracle.Tables(g, cb.cpu().numpy(), k, bits)
        assert T.total(k) == O.total(k)


def test_rebuild_replayed_from_a_cuda_graph(M):
    import torch
    k, bits = 5, 64
    g = synth.chung_lu_scaled(30000, seed=9)
    G = M.Graph.from_csr(g)
    cols = [M.color(G, k, 100 + i, out=torch.empty(g.n, dtype=torch.uint8, device="cuda"))
            for i in range(4)]
    buf = cols[0].clone()
    T = M.Tables(G, buf, k, bits)
    T.total(4)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up on the capture stream
        T.rebuild(buf)
    torch.cuda.current_stream().wait_stream(side)
    T.status()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        T.rebuild(buf)
    for i in (2, 1, 3):
        buf.copy_(cols[i])
        graph.replay()
        torch.cuda.synchronize()
        T.status()
        F = M.Tables(G, cols[i], k, bits)
        _same(T, F, k)


def test_rebuild_reports_bad_colours(M, oracle):
    import torch
    g = synth.er_1k()
    G = M.Graph.from_csr(g)
    good = M.color(G, 4, 0, out=torch.empty(g.n, dtype=torch.uint8, device="cuda"))
    T = M.Tables(G, good, 4, 64)
    bad = torch.full((g.n,), 9, dtype=torch.uint8, device="cuda")
    T.rebuild(bad)
    with pytest.raises(M.MotifError):
        T.status()
    with pytest.raises(M.MotifError):
        T.total(4)
    T.rebuild(good)
    T.status()
    O = oracle.Tables(g, good.cpu().numpy(), 4, 64)
    assert T.total(4) == O.total(4)
