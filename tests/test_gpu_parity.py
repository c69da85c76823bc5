"""Parity of the CUDA library (through its C ABI) with the CPU oracle.

Tables, neighbour sums, totals, colourings, samples and class ids must be
bit-exact; estimates (double) within 2 ulp.  Sizes span several warp tiles,
hubs (degree > 64, chunked paths) and ragged tails, plus the degenerate cases.
"""
import math

import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import layout

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    return M


def _oracle_tables(oracle, g, colors, k, bits):
    return oracle.Tables(g, colors, k, bits)


def assert_tables_equal(M, T, O, g, colors, k):
    """Every c and S entry of the GPU tables equals the oracle's."""
    for h in range(1, k + 1):
        r = cat.Catalog(k).r(h)
        gc = layout.gpu_c_as_oracle(T.read(h, 0), colors, k, h, r)
        oc = O.level(h)
        assert np.array_equal(gc, oc), f"c level {h}"
        if h <= k - 1:
            gs = layout.gpu_s_as_oracle(T.read(h, 1), colors, k, h, r)
            want = layout.neighbor_sums(oc, g.row_ptr, g.col)
            # S is stored only for sets without c_v
            mask = np.zeros(want.shape[:3], bool)
            idx = layout.s_index_map(k, h)[colors.astype(np.int64)]
            mask[np.arange(g.n)[:, None, None], np.arange(r)[None, :, None], idx[:, None, :]] = True
            want = np.where(mask[..., None], want, 0)
            assert np.array_equal(gs, want), f"S level {h}"


def assert_totals_equal(T, O, k):
    for h in range(1, k + 1):
        assert T.total(h) == O.total(h), h
        for j in range(len(cat.unrooted_shapes(h))):
            assert T.total(h, j) == O.total(h, j), (h, j)


def assert_samples_equal(T, O, h, seed, first, count, unrooted=-1):
    gn, gr, gs, gc = T.sample(h, seed, first, count, unrooted=unrooted)
    on, orr, os_, oc = O.sample(h, seed, first, count, unrooted=unrooted)
    assert np.array_equal(gn.cpu().numpy().astype(np.uint32), on)
    assert np.array_equal(gr.cpu().numpy().astype(np.uint32), orr)
    assert np.array_equal(gs.cpu().numpy(), os_)
    assert np.array_equal(gc.cpu().numpy(), oc)


CASES = [
    # (graph factory, k, bits, colouring seed)
    (lambda: synth.er_1k(), 4, 64, 0),                        # the 1k-node ER workload
    (lambda: synth.erdos_renyi(11, 4.0, seed=3), 2, 64, 1),
    (lambda: synth.erdos_renyi(12, 5.0, seed=4), 3, 64, 2),
    (lambda: synth.chung_lu_scaled(20000, seed=1), 5, 64, 3),  # hubs of up to ~700 neighbours
    (lambda: synth.chung_lu(5000, 30000, 2.3, seed=2), 6, 128, 4),
    (lambda: synth.erdos_renyi(1500, 7.0, seed=5), 7, 128, 5),
    (lambda: synth.erdos_renyi(300, 6.0, seed=6), 8, 128, 6),
    (lambda: synth.grid_road(40, seed=1), 5, 64, 7),
    (lambda: synth.lollipop(30, 6), 5, 128, 8),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tables_totals_samples(M, oracle, case):
    make, k, bits, cseed = CASES[case]
    g = make()
    colors = oracle.color(g.n, k, cseed)
    G = M.Graph.from_csr(g)
    gcol = M.color(G, k, cseed)
    assert np.array_equal(gcol.cpu().numpy(), colors)
    T = M.Tables(G, gcol, k, bits)
    O = oracle.Tables(g, colors, k, bits)
    assert_tables_equal(M, T, O, g, colors, k)
    assert_totals_equal(T, O, k)
    if T.total(k)[0] > 0:
        assert_samples_equal(T, O, k, seed=17 + case, first=0, count=3000)
        assert_samples_equal(T, O, k, seed=5, first=123_456_789_012, count=500)
    if k >= 4 and T.total(3)[0] > 0:
        assert_samples_equal(T, O, 3, seed=2, first=0, count=1000)
    for j in range(len(cat.unrooted_shapes(k))):
        if T.total(k, j)[0] > 0:
            assert_samples_equal(T, O, k, seed=9, first=0, count=500, unrooted=j)


@pytest.mark.parametrize("k,bits", [(4, 64), (5, 64), (6, 128)])
def test_zero_rooted_build(M, oracle, k, bits):
    g = synth.chung_lu_scaled(15000, seed=k)
    colors = oracle.color(g.n, k, 40 + k)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, colors, k, bits, zero_root=True)
    O = oracle.Tables(g, colors, k, bits, zero_root=True)
    assert_tables_equal(M, T, O, g, colors, k)
    assert_totals_equal(T, O, k)
    assert_samples_equal(T, O, k, seed=5, first=0, count=2000)
    for j in range(len(cat.unrooted_shapes(k))):
        if T.total(k, j)[0] > 0:
            assert_samples_equal(T, O, k, seed=6, first=0, count=300, unrooted=j)
    est, hits, _ = T.estimate(k, seed=2, samples=20000)
    oest, ohits = O.estimate_uniform(k, seed=2, n_samples=20000)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
    est, hits, st = T.estimate(k, seed=4, samples=200_000, mode=M.MC_EST_AGS, cbar=200)
    oest, ohits, ost = O.estimate_ags(k, seed=4, max_samples=200_000, cbar=200)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)


def test_k8_u128_with_hubs(M, oracle):
    """k = 8 with u128 counts on a power-law graph whose hubs (33 nodes of
    degree 65..140) take the chunked paths: the chunk-task gather, the hub
    reduction, and the sampler's search over hub chunk prefix sums."""
    g = synth.chung_lu(3000, 12000, 2.3, seed=11)
    assert int(g.degrees().max()) > 64
    k = 8
    colors = oracle.color(g.n, k, 9)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, M.color(G, k, 9), k, 128)
    O = oracle.Tables(g, colors, k, 128)
    assert_tables_equal(M, T, O, g, colors, k)
    assert_totals_equal(T, O, k)
    assert_samples_equal(T, O, k, seed=21, first=0, count=600)
    assert_samples_equal(T, O, k, seed=22, first=987_654_321, count=200)
    assert_samples_equal(T, O, 6, seed=23, first=0, count=300)   # h < k from the same tables
    for j in (0, 5, 11, len(cat.unrooted_shapes(k)) - 1):
        if T.total(k, j)[0] > 0:
            assert_samples_equal(T, O, k, seed=24, first=0, count=100, unrooted=j)
    est, hits, _ = T.estimate(k, seed=25, samples=2000)
    oest, ohits = O.estimate_uniform(k, seed=25, n_samples=2000)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)


def test_caller_colouring_and_device_csr(M, oracle):
    import torch
    g = synth.chung_lu(3000, 20000, 2.5, seed=9)
    colors = synth.random_colors(g.n, 5, seed=3)
    G = M.Graph(torch.as_tensor(g.row_ptr).cuda(), torch.as_tensor(g.col.astype(np.int32)).cuda())
    T = M.Tables(G, colors, 5, 64)
    O = oracle.Tables(g, colors, 5, 64)
    assert_tables_equal(M, T, O, g, colors, 5)


@pytest.mark.parametrize("h", range(1, 9))
def test_class_catalogue(M, oracle, h):
    assert M.num_classes(h) == oracle.num_classes(h)
    assert np.array_equal(M.class_codes(h), oracle.class_codes(h))
    si, sij = M.sigma(h)
    osi, osij = oracle.sigma(h)
    assert np.array_equal(si, osi)      # Kirchhoff (oracle) vs sum of the build's sigma_ij
    assert np.array_equal(sij, osij)


def _ulp_close(a, b, ulps=2):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    ia, ib = a.view(np.int64), b.view(np.int64)
    return bool(np.all(np.abs(ia - ib) <= ulps))


def test_uniform_estimates(M, oracle):
    g = synth.chung_lu_scaled(20000, seed=2)
    colors = oracle.color(g.n, 5, 1)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, colors, 5, 64)
    O = oracle.Tables(g, colors, 5, 64)
    est, hits, st = T.estimate(5, seed=3, samples=20000)
    oest, ohits = O.estimate_uniform(5, seed=3, n_samples=20000)
    assert np.array_equal(hits, ohits)
    assert _ulp_close(est, oest)
    assert st["samples"] == 20000


def test_ags_estimates(M, oracle):
    g = synth.chung_lu(4000, 24000, 2.3, seed=4)
    colors = oracle.color(g.n, 4, 2)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, colors, 4, 64)
    O = oracle.Tables(g, colors, 4, 64)
    # the run length per launch changes what is drawn ahead, never the result
    for batch, first in ((0, 0), (777, 0), (5000, 123_456_789)):
        est, hits, st = T.estimate(4, seed=8, samples=300_000, mode=M.MC_EST_AGS, cbar=300,
                                   batch=batch, first_index=first)
        oest, ohits, ost = O.estimate_ags(4, seed=8, max_samples=300_000, cbar=300, first_index=first)
        assert np.array_equal(hits, ohits)
        assert _ulp_close(est, oest)
        assert (st["samples"], st["switches"], st["covered"]) == \
            (ost["samples"], ost["switches"], ost["covered"])
    # every treelet's index stream holds 2^40 samples
    with pytest.raises(M.MotifError):
        T.estimate(4, seed=8, samples=(1 << 40) + 1, mode=M.MC_EST_AGS, cbar=300)


def test_overflow_is_reported(M, oracle):
    g = synth.star(1 << 16)
    colors = oracle.color(g.n, 6, 0)
    G = M.Graph.from_csr(g)
    with pytest.raises(M.MotifOverflow):
        M.Tables(G, colors, 6, 64)
    T = M.Tables(G, colors, 6, 128)
    O = oracle.Tables(g, colors, 6, 128)
    assert_tables_equal(M, T, O, g, colors, 6)


def test_degenerate_inputs(M, oracle):
    # no nodes
    G = M.Graph(np.zeros(1, np.int64), np.zeros(0, np.uint32))
    T = M.Tables(G, np.zeros(0, np.uint8), 4, 64)
    assert T.total(4) == (0, 0)
    with pytest.raises(M.MotifError):
        T.sample(4, 1, 0, 10)
    # isolated nodes only
    g = synth.from_edges(50, [], [])
    G = M.Graph.from_csr(g)
    T = M.Tables(G, oracle.color(50, 3, 0), 3, 64)
    assert T.total(3) == (0, 0) and T.total(1) == (50, 50)
    # zero samples is a no-op
    g = synth.er_1k()
    G = M.Graph.from_csr(g)
    T = M.Tables(G, oracle.color(g.n, 4, 0), 4, 64)
    T.sample(4, 1, 0, 0)
    # malformed graphs and colours are rejected
    with pytest.raises(M.MotifError):
        M.Graph(np.array([0, 1, 1], np.int64), np.array([1], np.uint32))      # asymmetric
    with pytest.raises(M.MotifError):
        M.Graph(np.array([0, 1, 2], np.int64), np.array([0, 0], np.uint32))   # loop
    with pytest.raises(M.MotifError):
        M.Graph(np.array([0, 2, 1], np.int64), np.array([1, 0], np.uint32))   # offsets
    with pytest.raises(M.MotifError):
        M.Tables(G, np.full(g.n, 7, np.uint8), 4, 64)
    with pytest.raises(M.MotifError):
        M.Tables(G, oracle.color(g.n, 9, 0), 9, 64)


@pytest.mark.parametrize("k,bits", [(5, 64), (7, 128)])
def test_small_and_large_launches_draw_the_same_samples(M, oracle, k, bits):
    """A launch too small to fill the GPU runs the sampler's latency mode
    (more loads in flight per lane, small blocks); a large one the throughput
    mode.  Sample i is the same either way: 100k samples in one launch equal
    the same indices drawn 4096 at a time, and the oracle's on a slice."""
    g = synth.chung_lu(20000, 150000, 2.3, seed=12)
    colors = oracle.color(g.n, k, 3)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, colors, k, bits)
    big = [x.cpu().numpy() for x in T.sample(k, 77, 1000, 100_000)]
    for first in (1000, 1000 + 4096 * 7, 1000 + 95_000):
        cnt = min(4096, 101_000 - first)
        small = [x.cpu().numpy() for x in T.sample(k, 77, first, cnt)]
        for a, b in zip(big, small):
            assert np.array_equal(a[first - 1000:first - 1000 + cnt], b)
    O = oracle.Tables(g, colors, k, bits)
    on, orr, osh, ocl = O.sample(k, 77, 1000 + 50_000, 300)
    assert np.array_equal(big[0][50_000:50_300].astype(np.uint32), on)
    assert np.array_equal(big[3][50_000:50_300], ocl)
