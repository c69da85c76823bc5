"""Parity at the benchmark's full size and launch configuration.

Chung-Lu n=1M, m~10M, exponent 2.5, k=5, 64-bit counts (the bench
workload) and the 1k-node Erdos-Renyi workload with k=4 and 10k samples.
Every count-table entry and total is compared with the oracle; neighbour
sums on sampled nodes (with the largest hubs), which the oracle computes one
by one; samples, classes and estimates bit for bit / within 2 ulp.
"""
import os

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import layout

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


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


def test_chung_lu_1m_k5_full_size(M, oracle):
    k, seed = 5, 12345
    g = synth.chung_lu_1m()
    G = M.Graph.from_csr(g)
    gcol = M.color(G, k, seed)
    colors = gcol.cpu().numpy()
    assert np.array_equal(colors, oracle.color(g.n, k, seed))
    T = M.Tables(G, gcol, k, 64)
    O = oracle.Tables(g, colors, k, 64, nthreads=os.cpu_count())
    C = cat.Catalog(k)
    for h in range(1, k + 1):
        gc = layout.gpu_c_as_oracle(T.read(h, 0), colors, k, h, C.r(h))
        assert np.array_equal(gc, O.level(h)), f"c level {h}"
        del gc
    for h in range(1, k + 1):
        assert T.total(h) == O.total(h)
        for j in range(len(cat.unrooted_shapes(h))):
            assert T.total(h, j) == O.total(h, j)
    # neighbour sums: the largest hubs and a random sample of nodes
    deg = g.degrees()
    rng = np.random.default_rng(0)
    nodes = np.unique(np.concatenate([np.argsort(deg)[-50:], rng.choice(g.n, 2000, replace=False)]))
    for h in range(1, k):
        gs = T.read(h, 1)
        Bs = layout.s_index_map(k, h)
        for v in nodes:
            want = O.neighbor_sum(h, int(v))            # [r, C(k,h), 2]
            got = gs[v].reshape(-1, C.r(h)).T          # set-major row -> [r, C(k-1,h)] u64
            idx = Bs[int(colors[v])]
            assert np.array_equal(got, want[:, idx, 0]) and not want[:, idx, 1].any(), (h, v)
    gn, gr, gsh, gcl = T.sample(k, seed=7, first_index=0, count=3000)
    on, orr, osh, ocl = O.sample(k, seed=7, first_index=0, count=3000)
    assert np.array_equal(gn.cpu().numpy().astype(np.uint32), on)
    assert np.array_equal(gr.cpu().numpy().astype(np.uint32), orr)
    assert np.array_equal(gsh.cpu().numpy(), osh)
    assert np.array_equal(gcl.cpu().numpy(), ocl)
    est, hits, _ = T.estimate(k, seed=9, samples=20_000)
    oest, ohits = O.estimate_uniform(k, seed=9, n_samples=20_000)
    assert np.array_equal(hits, ohits)
    assert _ulp_close(est, oest)


def test_er_1k_k4_10k_samples(M, oracle):
    k = 4
    g = synth.er_1k()
    G = M.Graph.from_csr(g)
    gcol = M.color(G, k, 0)
    colors = gcol.cpu().numpy()
    T = M.Tables(G, gcol, k, 64)
    O = oracle.Tables(g, colors, k, 64)
    gn, gr, gsh, gcl = T.sample(k, seed=1, first_index=0, count=10_000)
    on, orr, osh, ocl = O.sample(k, seed=1, first_index=0, count=10_000)
    assert np.array_equal(gn.cpu().numpy().astype(np.uint32), on)
    assert np.array_equal(gcl.cpu().numpy(), ocl)
    est, hits, _ = T.estimate(k, seed=1, samples=10_000)
    oest, ohits = O.estimate_uniform(k, seed=1, n_samples=10_000)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
    assert int(hits.sum()) == 10_000 and len(hits) == 6
