"""Serving with continuous batching: every request's result equals its
partition alone (and the oracle), admission keeps the running footprints
within the budget, and the footprint bound holds for every request."""
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402


@pytest.fixture(scope="module")
def mix():
    recipe = synth.batch_recipe(20, seed=7, log2_lo=8.0, log2_hi=13.0)
    host = [synth.batch_graph(s) for s in recipe]
    ks = [s["k"] for s in recipe]
    xr, ar = synth.rhg(1 << 14, 16.0, 2.8, 11)
    resident = tp.graph_from_csr(xr, ar).compress()
    return recipe, host, ks, (xr, ar), resident


def test_served_equals_alone(mix):
    recipe, host, ks, (xr, ar), resident = mix
    p = tp.default_params(seed=3)
    big = max(tp.footprint_bytes(len(x) - 1, len(a), k, True, True) for (x, a), k in zip(host, ks))
    with tp.Server(budget_bytes=3 * big, workers=4, params=p) as sv:
        tickets = []
        for i, ((x, a), k) in enumerate(zip(host, ks)):
            tickets.append(("host", i, sv.submit(k, 0.03, xadj=x, adj=a, compress=bool(i % 2))))
            if i % 4 == 0:  # requests on the resident graph, interleaved
                kr = (2, 8, 37, 256, 1024)[(i // 4) % 5]
                tickets.append(("res", kr, sv.submit(kr, 0.03, graph=resident)))
        results = [(kind, key, *sv.wait(t)) for kind, key, t in tickets]
        assert sv.peak_in_use() <= 3 * big
    for kind, key, part, st, info in results:
        assert info["peak_bytes"] <= info["footprint_bytes"], (kind, key, info)
        assert info["total_ms"] >= info["run_ms"] >= 0.0
        if kind == "host":
            x, a = host[key]
            g = tp.graph_from_csr(x, a)
            alone, ast = tp.partition(g, ks[key], 0.03, p)
            assert np.array_equal(part, alone.cpu().numpy()), key
            if key < 6:
                want, _ = oracle.partition(oracle.Graph(x, a), ks[key], 0.03, oracle.Params(seed=3))
                assert np.array_equal(part, want), key
        else:
            alone, ast = tp.partition(resident, key, 0.03, p)
            assert np.array_equal(part, alone.cpu().numpy()), key
        assert st["cut"] == ast["cut"]


def test_budget_admission(mix):
    recipe, host, ks, _, _ = mix
    fps = [tp.footprint_bytes(len(x) - 1, len(a), k) for (x, a), k in zip(host, ks)]
    budget = max(fps)  # the largest request only ever runs alone
    with tp.Server(budget_bytes=budget, workers=8) as sv:
        ts = [sv.submit(k, 0.03, xadj=x, adj=a) for (x, a), k in zip(host, ks)]
        infos = [sv.wait(t)[2] for t in ts]
        assert sv.peak_in_use() <= budget
        # a footprint beyond the whole budget: admitted alone, capped at the budget
        big = int(np.argmax(fps))
        x, a = host[big]
        part, _, info = sv.wait(sv.submit(ks[big], 0.03, xadj=x, adj=a, compress=True))
        assert info["footprint_bytes"] == budget and info["peak_bytes"] <= budget
        alone, _ = tp.partition(tp.graph_from_csr(x, a), ks[big], 0.03, tp.default_params())
        assert np.array_equal(part, alone.cpu().numpy())
        assert sv.peak_in_use() <= budget
    assert all(i["peak_bytes"] <= i["footprint_bytes"] for i in infos)


def test_ticket_is_waited_once(mix):
    recipe, host, ks, _, _ = mix
    x, a = host[-1]
    with tp.Server(budget_bytes=1 << 36, workers=2) as sv:
        t = sv.submit(ks[-1], 0.03, xadj=x, adj=a)
        # two waits on one ticket from two threads, through the C-ABI: exactly
        # one gets the request's status, the other TP_ERR_INVALID
        codes = []
        ths = [threading.Thread(target=lambda: codes.append(
            tp.lib().tp_server_wait(sv._h, t, None, None))) for _ in range(2)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        assert sorted(codes) == [0, 1]
        t2 = sv.submit(ks[0], 0.03, xadj=host[0][0], adj=host[0][1])
        part, _, _ = sv.wait(t2)
        with pytest.raises(tp.TpError):
            sv.wait(t2)


def test_footprint_bound_large_and_skewed():
    # the bound on graphs with very different shapes (hubs, random ids, locality)
    cases = [synth.rmat(15, 16, seed=2), synth.gnm(1 << 16, 1 << 19, 3),
             synth.rgg2d(1 << 17, 16.0, 4), synth.rhg(1 << 16, 32.0, 2.8, 5)]
    with tp.Server(budget_bytes=1 << 36, workers=2) as sv:
        for (x, a) in cases:
            for k, comp in ((2, False), (1024, True)):
                _, st, info = sv.wait(sv.submit(k, 0.03, xadj=x, adj=a, compress=comp))
                assert info["peak_bytes"] <= info["footprint_bytes"], (len(x) - 1, k, comp, info)
                assert st["balanced"]
