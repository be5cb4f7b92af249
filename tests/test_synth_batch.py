"""Input generators (CPU): the random hyperbolic generator against a direct
all-pairs test, the shapes of every generator (valid undirected CSR, sizes,
degrees, locality, skew, determinism) and the batch and serving recipes."""
import numpy as np
import pytest

import synth


def _csr_ok(xadj, adj):
    n = len(xadj) - 1
    deg = np.diff(xadj)
    src = np.repeat(np.arange(n), deg)
    assert not np.any(adj == src), "self-loop"
    for u in range(n):
        a = adj[xadj[u]:xadj[u + 1]]
        assert np.all(np.diff(a) > 0), "unsorted or duplicate"
    fwd = set(zip(src.tolist(), adj.tolist()))
    assert all((v, u) in fwd for u, v in fwd), "asymmetric"


@pytest.mark.parametrize("n,seed", [(64, 1), (700, 2), (3000, 3)])
def test_rhg_band_search_equals_all_pairs(n, seed):
    xa, aa = synth.rhg(n, 16.0, 2.8, seed)
    xb, ab = synth.rhg_brute(n, 16.0, 2.8, seed)
    assert np.array_equal(xa, xb) and np.array_equal(aa, ab)


def test_rhg_shape():
    n = 1 << 14
    xadj, adj = synth.rhg(n, 16.0, 2.8, 5)
    _csr_ok(xadj, adj)
    deg = np.diff(xadj)
    assert abs(len(adj) / n - 16.0) < 0.3  # calibrated average degree
    # heavy tail of a power law with exponent 2.8: hubs far above the mean,
    # and most vertices below it
    assert deg.max() > 20 * 16.0
    assert np.median(deg) < 16.0
    # same seed, same graph
    x2, a2 = synth.rhg(n, 16.0, 2.8, 5)
    assert np.array_equal(xadj, x2) and np.array_equal(adj, a2)


def test_batch_recipe():
    r = synth.batch_recipe(4096, seed=1)
    assert r == synth.batch_recipe(4096, seed=1)
    ns = np.array([s["n"] for s in r])
    assert ns.min() >= 256 and ns.max() <= 65536
    # log-uniform sizes: the median sits near 2^12
    assert 2 ** 11 < np.median(ns) < 2 ** 13
    assert [s["gen"] for s in r[:6]] == ["gnm", "rgg2d", "rhg"] * 2
    assert {s["k"] for s in r} == set(synth.BATCH_KS)
    assert len({s["seed"] for s in r}) == 4096
    for spec in r[:9]:
        xadj, adj = synth.batch_graph(spec)
        assert len(xadj) == spec["n"] + 1
        _csr_ok(xadj, adj)
        assert abs(len(adj) / spec["n"] - spec["deg"]) < 0.25 * spec["deg"]


def test_serving_recipe():
    import bench

    w = bench.WORKLOADS["serve"]
    r = bench.serve_recipe(w)
    assert r == bench.serve_recipe(w) and len(r) == w["count"]
    resident = [x for x in r if x["resident"]]
    assert len(resident) == w["count"] // 8  # every 8th request
    ks = [x["k"] for x in r]
    assert min(ks) >= 2 and max(ks) <= 1024 and len(set(ks)) > 20  # log-uniform over [2, 1024]
    ns = [x["n"] for x in r if not x["resident"]]
    assert min(ns) >= 2 ** w["log2_lo"] and max(ns) <= 2 ** w["log2_hi"]
    assert {x["gen"] for x in r if not x["resident"]} == set(synth.BATCH_GENERATORS)


def test_gnm_rgg_rmat_shapes():
    # G(n,m): exactly m distinct edges, ids without locality
    xadj, adj = synth.gnm(5000, 20000, 3)
    _csr_ok(xadj, adj)
    assert len(adj) == 2 * 20000
    # RGG-2D: expected degree d (a little less: points near the border lose
    # part of their disk), neighbour ids close to the vertex (cell order)
    n, d = 1 << 15, 16.0
    xadj, adj = synth.rgg2d(n, d, 4)
    _csr_ok(xadj, adj)
    assert 0.95 * d < len(adj) / n <= d
    src = np.repeat(np.arange(n), np.diff(xadj))
    assert np.median(np.abs(adj - src)) < n / 50
    # R-MAT scale 12, 16 samples per vertex: deduplicated and symmetrised
    # (so at most 2 * 16 * 2^12 entries), skewed towards low ids
    xadj, adj = synth.rmat(12, 16, seed=5)
    _csr_ok(xadj, adj)
    deg = np.diff(xadj)
    assert len(adj) <= 2 * 16 * 4096 and deg.max() > 20 * deg.mean()
    assert deg[: 4096 // 16].sum() > deg[-4096 // 16:].sum()
    # same seed, same graph; another seed, another graph
    assert np.array_equal(synth.gnm(5000, 20000, 3)[1], synth.gnm(5000, 20000, 3)[1])
    assert not np.array_equal(synth.gnm(5000, 20000, 3)[1], synth.gnm(5000, 20000, 4)[1])
