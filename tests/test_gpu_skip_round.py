"""Round skipping (MC_BUILD_SKIP_ROUND) and uncoloured star sampling on the
GPU against the oracle (Section 3.3.2).

Tables (every level but the skipped k-1, with level k built from balanced
decompositions), totals, samples, star samples and classes bit for bit;
uniform and adaptive estimates, with the star-only graphlet estimated from
uncoloured stars, within 2 ulp.
"""
import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests import layout
from tests.test_gpu_parity import _ulp_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    return M


CASES = [
    (lambda: synth.er_1k(), 4, 64, 0),
    (lambda: synth.chung_lu_scaled(20000, seed=1), 5, 64, 3),   # hubs, chunked paths
    (lambda: synth.chung_lu(5000, 30000, 2.3, seed=2), 6, 128, 4),
    (lambda: synth.chung_lu(3000, 15000, 2.4, seed=7), 7, 128, 5),
    (lambda: synth.erdos_renyi(300, 6.0, seed=6), 8, 128, 6),
    (lambda: synth.chung_lu(3000, 12000, 2.3, seed=11), 8, 128, 9),  # k = 8 with hubs (degree <= 140)
]


def _tables_equal_skipping(M, T, O, g, colors, k):
    C = cat.Catalog(k)
    for h in list(range(1, k - 1)) + [k]:
        gc = layout.gpu_c_as_oracle(T.read(h, 0), colors, k, h, C.r(h))
        assert np.array_equal(gc, O.level(h)), f"c level {h}"
    for h in range(1, k - 1):
        gs = layout.gpu_s_as_oracle(T.read(h, 1), colors, k, h, C.r(h))
        want = layout.neighbor_sums(O.level(h), g.row_ptr, g.col)
        mask = np.zeros(want.shape[:3], bool)
        idx = layout.s_index_map(k, h)[colors.astype(np.int64)]
        mask[np.arange(g.n)[:, None, None], np.arange(C.r(h))[None, :, None], idx[:, None, :]] = True
        assert np.array_equal(gs, np.where(mask[..., None], want, 0)), f"S level {h}"
    for which in (0, 1):
        with pytest.raises(M.MotifError):
            T.read(k - 1, which)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_skip_round_against_oracle(M, oracle, case):
    make, k, bits, cseed = CASES[case]
    g = make()
    colors = oracle.color(g.n, k, cseed)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, colors, k, bits, skip_round=True)
    O = oracle.Tables(g, colors, k, bits, skip_round=True)
    _tables_equal_skipping(M, T, O, g, colors, k)
    for h in list(range(1, k - 1)) + [k]:
        assert T.total(h) == O.total(h), h
        for j in range(len(cat.unrooted_shapes(h))):
            assert T.total(h, j) == O.total(h, j), (h, j)
    with pytest.raises(M.MotifError):
        T.total(k - 1)
    with pytest.raises(M.MotifError):
        T.sample(k - 1, 1, 0, 10)
    n_s = 3000 if k < 8 else 1000
    if T.total(k)[0] > 0:
        for seed, first, count in ((17, 0, n_s), (5, 123_456_789, 500)):
            gn, gr, gs, gc = T.sample(k, seed, first, count)
            on, orr, os_, oc = O.sample(k, seed, first, count)
            assert np.array_equal(gn.cpu().numpy().astype(np.uint32), on)
            assert np.array_equal(gr.cpu().numpy().astype(np.uint32), orr)
            assert np.array_equal(gs.cpu().numpy(), os_)
            assert np.array_equal(gc.cpu().numpy(), oc)
    hs = 3 if k > 4 else 2  # a level below the skipped one
    gn, gr, gs, gc = T.sample(hs, 2, 0, 1000)
    on, orr, os_, oc = O.sample(hs, 2, 0, 1000)
    assert np.array_equal(gn.cpu().numpy().astype(np.uint32), on)
    assert np.array_equal(gc.cpu().numpy(), oc)
    # uncoloured k-stars
    assert G.star_total(k) == O.star_total(k)
    if O.star_total(k) > 0:
        sn, sc, scl = G.sample_stars(k, 9, 77, n_s)
        on, oc, ocl = O.sample_stars(k, 9, 77, n_s)
        assert np.array_equal(sn.cpu().numpy().astype(np.uint32), on)
        assert np.array_equal(sc.cpu().numpy().astype(np.uint32), oc)
        assert np.array_equal(scl.cpu().numpy(), ocl)
    # estimates (the oracle classifies an 8-node sample by trying all 8!
    # relabelings, so k = 8 takes fewer samples)
    n_uni, n_ags, n_star, cbar = (20000, 100_000, 5000, 100) if k < 8 else (2000, 4000, 1000, 20)
    if T.total(k)[0] > 0:
        est, hits, _ = T.estimate(k, seed=3, samples=n_uni, star_samples=n_star)
        oest, ohits = O.estimate_uniform(k, seed=3, n_samples=n_uni, star_samples=n_star)
        assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
        est, hits, st = T.estimate(k, seed=4, samples=n_ags, mode=M.MC_EST_AGS, cbar=cbar,
                                   star_samples=n_star)
        oest, ohits, ost = O.estimate_ags(k, seed=4, max_samples=n_ags, cbar=cbar,
                                          star_samples=n_star)
        assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
        assert (st["samples"], st["switches"], st["covered"]) == \
            (ost["samples"], ost["switches"], ost["covered"])


def test_skip_round_rejects_bad_combinations(M, oracle):
    g = synth.er_1k()
    G = M.Graph.from_csr(g)
    colors = oracle.color(g.n, 4, 0)
    with pytest.raises(M.MotifError):
        M.Tables(G, colors, 4, 64, skip_round=True, zero_root=True)
    with pytest.raises(M.MotifError):
        M.Tables(G, oracle.color(g.n, 3, 0), 3, 64, skip_round=True)
    P = M.Graph.from_csr(synth.path(50))       # maximum degree 2: no 4-star
    assert P.star_total(4) == 0 and P.star_total(3) == 48
    with pytest.raises(M.MotifError):
        P.sample_stars(4, 1, 0, 10)


def test_skip_round_equals_full_build_below(M, oracle):
    # levels 1..k-2 and the non-star level-k totals are those of the full build
    g = synth.chung_lu_scaled(30000, seed=4)
    colors = oracle.color(g.n, 6, 1)
    G = M.Graph.from_csr(g)
    A = M.Tables(G, colors, 6, 128)
    Z = M.Tables(G, colors, 6, 128, skip_round=True)
    for h in range(1, 5):
        assert np.array_equal(A.read(h, 0), Z.read(h, 0))
    star = cat.unrooted_id("10" * 5)
    for j in range(len(cat.unrooted_shapes(6))):
        assert Z.total(6, j)[1] == (0 if j == star else A.total(6, j)[1])
