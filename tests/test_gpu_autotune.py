"""Every schedule the autotuner can pick computes the same exact tables.

Each neighbour-sum schedule (0..6) and each merge schedule (0..5) is pinned
in turn for every level of a build (mc_autotune_set, tuning off), and the
tables must equal the oracle's bit for bit: at k = 5 with u64 counts (8- and
16-byte units, 2 to 8 lanes per node) and k = 6 with u128 counts (up to 32
lanes per node), on graphs with hubs.
"""
import numpy as np
import pytest

import synth
from oracle import catalog as cat
from tests.test_gpu_parity import assert_tables_equal, assert_totals_equal

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    yield M
    M.autotune(1)


@pytest.mark.parametrize("k,bits,make", [
    (5, 64, lambda: synth.chung_lu_scaled(20000, seed=8)),
    (6, 128, lambda: synth.chung_lu(5000, 30000, 2.3, seed=9)),
])
def test_every_schedule_builds_the_same_tables(M, oracle, k, bits, make):
    g = make()
    colors = oracle.color(g.n, k, 31)
    O = oracle.Tables(g, colors, k, bits)
    G = M.Graph.from_csr(g)
    n, nnz, maxd = G.info()
    M.autotune(0)  # pinned choices only
    for gs, ms in [(0, 0), (1, 1), (2, 2), (3, 3), (4, 4), (5, 5), (6, 0)]:
        for h in range(2, k + 1):
            M.autotune_set(1, k, bits, h, n, nnz, maxd, ms)
            if h < k:
                M.autotune_set(0, k, bits, h, n, nnz, maxd, gs)
        T = M.Tables(G, colors, k, bits)
        assert_tables_equal(M, T, O, g, colors, k)
        assert_totals_equal(T, O, k)
        for h in range(2, k):
            assert M.autotune_choice(0, k, bits, h, n, nnz, maxd) == gs
        T.free()


def test_tuning_keeps_results(M, oracle):
    # a forced re-tune times every schedule; the tables stay the oracle's
    g = synth.chung_lu_scaled(20000, seed=10)
    k = 5
    colors = oracle.color(g.n, k, 5)
    G = M.Graph.from_csr(g)
    M.autotune(2)
    T = M.Tables(G, colors, k, 64)
    M.autotune(1)
    O = oracle.Tables(g, colors, k, 64)
    assert_tables_equal(M, T, O, g, colors, k)
    n, nnz, maxd = G.info()
    for h in range(2, k):
        assert 0 <= M.autotune_choice(0, k, 64, h, n, nnz, maxd) < 7
    for h in range(2, k + 1):
        assert 0 <= M.autotune_choice(1, k, 64, h, n, nnz, maxd) < 6
