"""Biased colouring (Section 3.5) and non-zero entry counts on the GPU
against the oracle: colours bit for bit, tables and samples bit for bit,
uniform and adaptive estimates with the biased colourful probability within
2 ulp; non-zero counts equal those of the oracle's tables."""
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


@pytest.mark.parametrize("k,L", [(4, 3 * 2**28), (5, 2**29 + 12345), (8, 12_345_678)])
def test_biased_colours(M, oracle, k, L):
    g = synth.chung_lu_scaled(50000, seed=k)
    G = M.Graph.from_csr(g)
    got = M.color(G, k, 11, bias_q32=L).cpu().numpy()
    assert np.array_equal(got, oracle.color_biased(g.n, k, 11, L))
    with pytest.raises(M.MotifError):
        M.color(G, k, 1, bias_q32=2**32 // (k - 1) + 1)


@pytest.mark.parametrize("k,bits,L", [(5, 64, 2**29 + 12345), (6, 128, 3 * 2**27)])
def test_biased_tables_and_estimates(M, oracle, k, bits, L):
    g = synth.chung_lu(20000, 150000, 2.3, seed=k)
    G = M.Graph.from_csr(g)
    gcol = M.color(G, k, 5, bias_q32=L)
    colors = gcol.cpu().numpy()
    T = M.Tables(G, gcol, k, bits)
    O = oracle.Tables(g, colors, k, bits)
    C = cat.Catalog(k)
    for h in range(1, k + 1):
        oc = O.level(h)
        assert np.array_equal(layout.gpu_c_as_oracle(T.read(h, 0), colors, k, h, C.r(h)), oc)
        nz = int(np.count_nonzero(oc.any(axis=-1)))
        assert T.nonzeros(h) == nz, h
        assert T.total(h) == O.total(h)
    for h in range(1, k):
        S = layout.gpu_s_as_oracle(T.read(h, 1), colors, k, h, C.r(h))
        assert T.nonzeros(h, 1) == int(np.count_nonzero(S.any(axis=-1)))
    if T.total(k)[0] == 0:
        return
    gn, _, _, gc = T.sample(k, 3, 0, 2000)
    on, _, _, oc = O.sample(k, 3, 0, 2000)
    assert np.array_equal(gn.cpu().numpy().astype(np.uint32), on)
    assert np.array_equal(gc.cpu().numpy(), oc)
    est, hits, _ = T.estimate(k, seed=4, samples=20000, colour_bias_q32=L)
    oest, ohits = O.estimate_uniform(k, seed=4, n_samples=20000, bias_q32=L)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
    est, hits, st = T.estimate(k, seed=6, samples=100_000, mode=M.MC_EST_AGS, cbar=100,
                               colour_bias_q32=L)
    oest, ohits, ost = O.estimate_ags(k, seed=6, max_samples=100_000, cbar=100, bias_q32=L)
    assert np.array_equal(hits, ohits) and _ulp_close(est, oest)
    # the uniform colouring's probability is a different number
    est0, _, _ = T.estimate(k, seed=4, samples=20000)
    assert not np.array_equal(est0, T.estimate(k, seed=4, samples=20000, colour_bias_q32=L)[0])
