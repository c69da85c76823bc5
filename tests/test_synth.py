"""The seeded input generators: canonical CSR, determinism, and the shape
of the stand-in workloads (degree exponent and cut-off, average degree,
R-MAT skew)."""
import numpy as np

import synth


def _canonical(g):
    rp, col = g.row_ptr, g.col.astype(np.int64)
    assert rp[0] == 0 and rp[-1] == len(col) and np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    assert np.all(src != col)                                     # no loops
    for v in range(min(g.n, 200)):                                # sorted, no duplicates
        assert np.all(np.diff(col[rp[v]:rp[v + 1]]) > 0)
    a = np.sort(src * g.n + col)
    b = np.sort(col * g.n + src)
    assert np.array_equal(a, b)                                   # symmetric


def test_generators_are_canonical_and_seeded():
    for make in (lambda s: synth.erdos_renyi(500, 6.0, seed=s),
                 lambda s: synth.chung_lu(3000, 20000, 2.5, seed=s),
                 lambda s: synth.rmat(11, 8, seed=s),
                 lambda s: synth.grid_road(20, seed=s)):
        g1, g2, g3 = make(1), make(1), make(2)
        _canonical(g1)
        assert np.array_equal(g1.col, g2.col) and np.array_equal(g1.row_ptr, g2.row_ptr)
        assert not (len(g1.col) == len(g3.col) and np.array_equal(g1.col, g3.col))


def test_erdos_renyi_average_degree():
    g = synth.erdos_renyi(20000, 8.0, seed=0)
    assert abs(g.degrees().mean() - 8.0) < 0.1


def test_chung_lu_exponent_and_cutoff():
    # the degree CCDF of a power law with exponent gamma falls as d^(1 - gamma)
    n, m, gamma = 200_000, 2_000_000, 2.5
    g = synth.chung_lu(n, m, gamma, max_degree=2000.0, seed=3)
    d = g.degrees()
    assert 0.97 * m < g.m <= m                      # loops and duplicates dropped
    assert 1500 < d.max() < 2600                    # the requested cut-off
    xs = np.array([40, 80, 160, 320])
    ccdf = np.array([(d >= x).mean() for x in xs])
    slope = np.polyfit(np.log(xs), np.log(ccdf), 1)[0]
    assert abs(slope - (1 - gamma)) < 0.2, slope


def test_rmat_skew():
    # quadrant probabilities .57/.19/.19/.05 make a heavy-tailed degree
    # sequence: the top 1% of nodes hold far more than 1% of the edges
    g = synth.rmat(14, 16, seed=0)
    d = np.sort(g.degrees())[::-1]
    assert d[: g.n // 100].sum() > 0.1 * d.sum()
    # edge factor 16: 16 n generated edges, loops and duplicates dropped
    assert 0.75 * 16 * g.n < g.m <= 16 * g.n
