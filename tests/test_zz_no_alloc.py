"""The uniform estimator's no-allocation entry point, through the C ABI.

Some callers cannot allocate device memory at the moment they need an
estimate: code running under CUDA stream capture (cudaMalloc is illegal
there), serving loops whose memory is all owned by a pool reserved up
front, and latency-critical loops that cannot afford cudaMalloc's implicit
device synchronisation.  mc_estimate_uniform_noalloc serves them with a
static device scratch array; its results must equal those of
mc_estimate_counts in uniform mode (hits exactly, estimates within 2 ulp),
call after call, since every call reuses and re-clears the same scratch.

This file is collected last so that a failure here stops a -x run only
after every other test has run.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _ulp_close(a, b, ulps=2):
    ia = np.asarray(a, np.float64).view(np.int64)
    ib = np.asarray(b, np.float64).view(np.int64)
    return bool(np.all(np.abs(ia - ib) <= ulps))


def test_noalloc_estimate_matches_allocating_estimate():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    k = 5
    g = synth.chung_lu_scaled(20000, seed=3)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, M.color(G, k, 11), k, 64)
    M.sigma(k)  # the catalogue must exist before the no-allocation call
    for seed, first in ((21, 0), (22, 1000)):  # two calls in a row share the scratch
        est, hits = T.estimate_noalloc(k, seed, 40_000, first_index=first)
        est2, hits2, st = T.estimate(k, seed=seed, samples=40_000, first_index=first)
        assert int(hits.sum()) == 40_000
        assert np.array_equal(hits, hits2)
        assert _ulp_close(est, est2)
