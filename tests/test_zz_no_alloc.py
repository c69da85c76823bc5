"""The uniform estimator's no-allocation entry point, through the C ABI.

Some callers cannot allocate device memory at the moment they need an
estimate: serving loops whose device memory is all owned by a pool reserved
up front, and latency-critical loops that cannot afford cudaMalloc's
implicit device synchronisation.  mc_estimate_uniform_noalloc serves them
with a static device scratch array; its results must equal those of
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


def _lib():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    return M


def test_noalloc_estimate_matches_allocating_estimate():
    M = _lib()
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


def test_noalloc_refuses_a_lower_level_index_older_than_a_rebuild():
    """A root index of a level below k belongs to the colouring it was made
    for: after an in-place rebuild the call refuses it (remaking it would
    allocate) until mc_total remakes it, and then matches the allocating
    estimate again."""
    M = _lib()
    k, h = 5, 4
    g = synth.chung_lu_scaled(20000, seed=5)
    G = M.Graph.from_csr(g)
    T = M.Tables(G, M.color(G, k, 1), k, 64)
    M.sigma(h)
    T.total(h)  # makes the level-4 root index
    est, hits = T.estimate_noalloc(h, 31, 20_000)
    est2, hits2, _ = T.estimate(h, seed=31, samples=20_000)
    assert np.array_equal(hits, hits2) and _ulp_close(est, est2)
    T.rebuild(M.color(G, k, 2))
    with pytest.raises(M.MotifError) as e:  # before mc_tables_status: the whole tables are stale
        T.estimate_noalloc(h, 31, 20_000)
    assert e.value.status == M.MC_E_INVALID
    T.status()
    with pytest.raises(M.MotifError) as e:  # level 4's index is from the first colouring
        T.estimate_noalloc(h, 31, 20_000)
    assert e.value.status == M.MC_E_INVALID
    T.total(h)
    for seed in (32, 33):
        est, hits = T.estimate_noalloc(h, seed, 20_000)
        est2, hits2, _ = T.estimate(h, seed=seed, samples=20_000)
        assert int(hits.sum()) == 20_000
        assert np.array_equal(hits, hits2)
        assert _ulp_close(est, est2)
    # level k's index is rebuilt with the tables: usable right after the status check
    est, hits = T.estimate_noalloc(k, 34, 20_000)
    est2, hits2, _ = T.estimate(k, seed=34, samples=20_000)
    assert np.array_equal(hits, hits2) and _ulp_close(est, est2)
