"""Batched builds (many colourings of one graph plus many graphs of uneven
sizes, k = 6, 128-bit counts) against the plain single-instance path and
the oracle: every count, total, sample and estimate of an instance must be
identical whether it was built alone or inside the batch."""
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


def _instances(oracle, k):
    base = synth.chung_lu(20000, 200000, 2.3, seed=5)
    inst = [(base, oracle.color(base.n, k, 100 + i)) for i in range(6)]
    rng = np.random.default_rng(1)
    for i in range(6):
        n = int(np.exp(rng.uniform(np.log(1000), np.log(10000))))
        deg = float(rng.uniform(4, 20))
        g = synth.erdos_renyi(n, deg, seed=i) if i % 2 == 0 else synth.chung_lu(n, int(n * deg / 2), 2.3, seed=i)
        inst.append((g, oracle.color(g.n, k, 200 + i)))
    return inst


def test_batch_equals_single_instances(M, oracle):
    k, bits = 6, 128
    inst = _instances(oracle, k)
    graphs = [M.Graph.from_csr(g) for g, _ in inst]
    TB, offs = M.Tables.batch(graphs, [c for _, c in inst], k, bits)
    assert offs[-1] == sum(g.n for g, _ in inst)
    for i, ((g, col), G) in enumerate(zip(inst, graphs)):
        lo, hi = int(offs[i]), int(offs[i + 1])
        T = M.Tables(G, col, k, bits)
        for h in range(1, k + 1):
            assert TB.total(h, node_range=(lo, hi)) == T.total(h), (i, h)
            for j in range(len(cat.unrooted_shapes(h))):
                assert TB.total(h, j, node_range=(lo, hi)) == T.total(h, j)
            # the tables themselves: instance i's rows of the union
            a = TB.read(h, 0)[lo:hi]
            assert np.array_equal(a, T.read(h, 0))
        if T.total(k)[0] == 0:
            continue
        bn, br, bs, bc = TB.sample(k, 31 + i, 0, 1000, node_range=(lo, hi))
        sn, sr, ss, sc = T.sample(k, 31 + i, 0, 1000)
        assert np.array_equal(bn.cpu().numpy() - lo, sn.cpu().numpy())
        assert np.array_equal(br.cpu().numpy() - lo, sr.cpu().numpy())
        assert np.array_equal(bs.cpu().numpy(), ss.cpu().numpy())
        assert np.array_equal(bc.cpu().numpy(), sc.cpu().numpy())
        be, bh, _ = TB.estimate(k, seed=9, samples=20000, node_range=(lo, hi))
        se, sh, _ = T.estimate(k, seed=9, samples=20000)
        assert np.array_equal(bh, sh) and np.array_equal(be, se)
    # one batch instance straight against the oracle, AGS included
    i = 7
    g, col = inst[i]
    lo, hi = int(offs[i]), int(offs[i + 1])
    O = oracle.Tables(g, col, k, bits)
    bn, _, _, bc = TB.sample(k, 5, 0, 1000, node_range=(lo, hi))
    on, _, _, oc = O.sample(k, 5, 0, 1000)
    assert np.array_equal(bn.cpu().numpy().astype(np.uint32) - lo, on)
    assert np.array_equal(bc.cpu().numpy(), oc)
    be, bh, st = TB.estimate(k, seed=4, samples=100_000, mode=M.MC_EST_AGS, cbar=100,
                             node_range=(lo, hi))
    oe, oh, ost = O.estimate_ags(k, seed=4, max_samples=100_000, cbar=100)
    assert np.array_equal(bh, oh)
    assert (st["samples"], st["switches"]) == (ost["samples"], ost["switches"])


def test_union_rebuild_replayed_from_a_cuda_graph(M, oracle):
    """The whole batch rebuilt in place for new colourings of every instance:
    one captured CUDA graph of mc_rebuild_tables on the union, replayed; each
    instance's rows then equal a fresh single build with its new colouring."""
    import torch
    k, bits = 6, 128
    inst = _instances(oracle, k)
    graphs = [M.Graph.from_csr(g) for g, _ in inst]
    TB, offs = M.Tables.batch(graphs, [c for _, c in inst], k, bits)
    buf = torch.empty(int(offs[-1]), dtype=torch.uint8, device="cuda")
    s = torch.cuda.current_stream()
    side = torch.cuda.Stream()
    side.wait_stream(s)
    with torch.cuda.stream(side):
        TB.rebuild(torch.cat([torch.as_tensor(c).cuda() for _, c in inst]))
    s.wait_stream(side)
    TB.status()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        TB.rebuild(buf)
    for rnd in range(2):
        new = [oracle.color(g.n, k, 900 + 10 * rnd + i) for i, (g, _) in enumerate(inst)]
        buf.copy_(torch.cat([torch.as_tensor(c) for c in new]).cuda())
        graph.replay()
        TB.status()
        for i, (G, c) in enumerate(zip(graphs, new)):
            lo, hi = int(offs[i]), int(offs[i + 1])
            T = M.Tables(G, c, k, bits)
            for h in (2, 4, k):
                assert np.array_equal(TB.read(h, 0)[lo:hi], T.read(h, 0)), (rnd, i, h)
            assert TB.total(k, node_range=(lo, hi)) == T.total(k)
