"""tp_footprint_bytes against what partitions actually hold at their peak
(stats peak_bytes), on the graph classes of the benchmarks: skewed R-MAT,
hyperbolic (power-law) graphs with average degree 16 and 32, geometric and
uniform random graphs, CSR and compressed; and the server's enforcement of
footprints (a request that outgrows its footprint runs again alone)."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402

CASES = [
    ("rmat22", lambda: synth.rmat(22, 16, seed=1), 256),
    ("rmat24", lambda: synth.rmat(24, 16, seed=1), 256),
    ("rhg20_d16", lambda: synth.rhg(1 << 20, 16.0, 2.8, 3), 64),
    ("rhg20_d32", lambda: synth.rhg(1 << 20, 32.0, 2.8, 4), 1024),
    ("rgg22", lambda: synth.rgg2d(1 << 22, 16.0, 5), 64),
    ("gnm20", lambda: synth.gnm(1 << 20, 8 << 20, 6), 8),
]


@pytest.mark.parametrize("name,make,k", CASES, ids=[c[0] for c in CASES])
def test_peak_within_footprint(name, make, k):
    xadj, adj = make()
    n, m2 = len(xadj) - 1, len(adj)
    g = tp.graph_from_csr(xadj, adj)
    bound = tp.footprint_bytes(n, m2, k, upload=False, compress=False)
    for gg in (g.compress(), g):
        _, st = tp.partition(gg, k, 0.03, tp.default_params(seed=1))
        assert 0 < st["peak_bytes"] <= bound, (name, st["peak_bytes"], bound)
    # uploading (and compressing) through the server stays inside its figure too
    with tp.Server(budget_bytes=tp.footprint_bytes(n, m2, k, True, True), workers=1) as sv:
        _, _, info = sv.wait(sv.submit(k, 0.03, xadj=xadj, adj=adj, compress=True))
        assert info["retries"] == 0 and info["peak_bytes"] <= info["footprint_bytes"]


def test_request_outgrowing_its_footprint_runs_again_alone(monkeypatch):
    """Footprints scaled down to 2% are too small: every request fails before
    allocating beyond its share, runs again alone with the whole budget, and
    its result is still the one it has alone; the budget is never exceeded."""
    monkeypatch.setenv("TP_FOOTPRINT_SCALE", "0.02")
    recipe = synth.batch_recipe(8, seed=9, log2_lo=12.0, log2_hi=15.0)
    host = [synth.batch_graph(s) for s in recipe]
    ks = [s["k"] for s in recipe]
    budget = 2 * max(tp.footprint_bytes(len(x) - 1, len(a), k) for (x, a), k in zip(host, ks))
    p = tp.default_params(seed=2)
    with tp.Server(budget_bytes=budget, workers=4, params=p) as sv:
        ts = [sv.submit(k, 0.03, xadj=x, adj=a) for (x, a), k in zip(host, ks)]
        res = [sv.wait(t) for t in ts]
        assert sv.peak_in_use() <= budget
    assert any(info["retries"] == 1 for _, _, info in res)
    for ((x, a), k), (part, st, info) in zip(zip(host, ks), res):
        alone, _ = tp.partition(tp.graph_from_csr(x, a), k, 0.03, p)
        assert np.array_equal(part, alone.cpu().numpy())
        assert info["peak_bytes"] <= info["footprint_bytes"]
        if info["retries"]:
            assert info["footprint_bytes"] == budget
