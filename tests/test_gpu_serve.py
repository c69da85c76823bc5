"""The serving loop (mc_server_*): a mix of sample and estimate requests of
different sizes, treelet sizes and tables, submitted together and run
concurrently on several slots, must give for every request exactly what the
same request gives alone; with a tiny memory budget requests queue for
admission and the results are still the same."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    import paper_2009_03052_gb300 as M
    M.build()
    M.load()
    g1 = synth.chung_lu_scaled(30000, seed=3)
    g2 = synth.erdos_renyi(6000, 8.0, seed=4)
    G1, G2 = M.Graph.from_csr(g1), M.Graph.from_csr(g2)
    T1 = M.Tables(G1, M.color(G1, 5, 1), 5, 64, own_memory=True)
    T2 = M.Tables(G2, M.color(G2, 6, 2), 6, 128, own_memory=True)
    for h in (3, 4, 5):
        M.sigma(h)
    return M, [T1, T2], (G1, G2)


def _mix():
    rng = np.random.default_rng(11)
    reqs = []
    for i in range(24):
        t = i % 2
        k = 5 if t == 0 else 6
        kind = ["sample", "sample", "uniform", "ags"][i % 4]
        if kind == "sample":
            reqs.append(("sample", t, int(rng.integers(3, k + 1)), 100 + i,
                         int(np.exp(rng.uniform(np.log(1e3), np.log(2e5))))))
        elif kind == "uniform":
            reqs.append(("uniform", t, int(rng.integers(3, 6)), 200 + i, 50_000))
        else:
            reqs.append(("ags", t, 4, 300 + i, 100_000))
    return reqs


def _alone(M, T, r):
    kind, t, h, seed, n = r
    if kind == "sample":
        nodes, _, _, cls = T[t].sample(h, seed, 0, n, roots=False, shapes=False)
        return nodes.cpu().numpy().astype(np.uint32), cls.cpu().numpy()
    mode = M.MC_EST_UNIFORM if kind == "uniform" else M.MC_EST_AGS
    est, hits, _ = T[t].estimate(h, seed, n, mode=mode, cbar=100)
    return est, hits


def _submit(M, S, r):
    kind, t, h, seed, n = r
    if kind == "sample":
        return S.submit_sample(t, h, seed, n)
    mode = M.MC_EST_UNIFORM if kind == "uniform" else M.MC_EST_AGS
    return S.submit_estimate(t, h, seed, n, mode=mode, cbar=100)


def _check(r, res, want):
    if r[0] == "sample":
        assert np.array_equal(res["nodes"], want[0]) and np.array_equal(res["classes"], want[1]), r
    else:
        assert np.array_equal(res["hits"], want[1]) and np.array_equal(res["est"], want[0]), r
    assert 0 <= res["queue_us"] <= res["latency_us"]


def test_each_result_is_the_same_alone_and_in_the_mix(setup):
    M, T, _ = setup
    reqs = _mix()
    want = [_alone(M, T, r) for r in reqs]
    S = M.Server(T, slots=4)
    ids = [_submit(M, S, r) for r in reqs]
    for r, i, w in zip(reqs, ids, want):
        _check(r, S.wait(i), w)
    # requests submitted while others run
    ids = []
    for j, r in enumerate(reqs):
        ids.append(_submit(M, S, r))
        if j % 5 == 4:
            _check(reqs[j - 4], S.wait(ids[j - 4]), want[j - 4])
            ids[j - 4] = None
    for r, i, w in zip(reqs, ids, want):
        if i is not None:
            _check(r, S.wait(i), w)
    S.free()


def test_tiny_budget_queues_requests_with_the_same_results(setup):
    M, T, _ = setup
    reqs = _mix()[:8]
    want = [_alone(M, T, r) for r in reqs]
    S = M.Server(T, slots=3, memory_budget=1)  # every request needs more: one at a time
    ids = [_submit(M, S, r) for r in reqs]
    res = [S.wait(i) for i in ids]
    for r, x, w in zip(reqs, res, want):
        _check(r, x, w)
    assert max(x["queue_us"] for x in res) > 0
    S.free()


@pytest.mark.slow
def test_serving_workload_full_size(oracle):
    # Chung-Lu n = 2M, m ~ 20M, k = 8, 128-bit counts: star totals by their
    # closed form at every level; samples of sizes 5..8 drawn through the
    # server are the same as drawn directly, and each is colourful,
    # connected and carries the oracle's class of its induced subgraph
    import torch
    import paper_2009_03052_gb300 as M
    from oracle import catalog as cat
    from tests import brute
    k = 8
    g = synth.chung_lu(2_000_000, 20_000_000, 2.5, max_degree=10_000.0, seed=0)
    G = M.Graph.from_csr(g, trusted=True)
    col = M.color(G, k, 1)
    colors = col.cpu().numpy()
    T = M.Tables(G, col, k, 128, own_memory=True)
    stars = brute.star_totals(g, colors, k)
    assert T.total(2)[1] == stars[2]
    for h in range(3, k + 1):
        assert T.total(h, cat.unrooted_id("10" * (h - 1)))[1] == stars[h], h
    S = M.Server([T], slots=4)
    ids = [(h, S.submit_sample(0, h, 50 + h, 500)) for h in (5, 6, 7, 8)]
    for h, rid in ids:
        res = S.wait(rid)
        nodes, _, _, cls = T.sample(h, 50 + h, 0, 500, roots=False, shapes=False)
        nodes = nodes.cpu().numpy().astype(np.uint32)
        assert np.array_equal(res["nodes"], nodes) and np.array_equal(res["classes"], cls.cpu().numpy())
        for s in range(0, 500, 5):
            vs = nodes[s].astype(np.int64)
            assert len(set(colors[vs].tolist())) == h
            w = 0
            for a in range(h):
                row = g.col[g.row_ptr[vs[a]]:g.row_ptr[vs[a] + 1]]
                for b in range(a + 1, h):
                    i = np.searchsorted(row, vs[b])
                    w = (w << 1) | int(i < len(row) and row[i] == vs[b])
            assert res["classes"][s] == oracle.class_of_word(h, w) >= 0
    S.free()
    T.free()
    torch.cuda.synchronize()
