"""Batched mode: every graph of a batch equals its single-graph partition and
the oracle, whatever the stream count and the tuned performance knobs."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402
from paper_2410_19119_gb300 import autotune  # noqa: E402


@pytest.fixture(scope="module")
def small_batch():
    # the batch recipe at sizes the oracle finishes quickly (n <= 2^11.5)
    recipe = synth.batch_recipe(36, seed=3, log2_lo=8.0, log2_hi=11.5)
    csr = [synth.batch_graph(s) for s in recipe]
    graphs = []
    for i, (xadj, adj) in enumerate(csr):
        g = tp.graph_from_csr(xadj, adj)
        graphs.append(g.compress() if i % 2 else g)  # both storage formats in one batch
    return recipe, csr, graphs


def test_batch_equals_single_and_oracle(small_batch):
    recipe, csr, graphs = small_batch
    ks = [s["k"] for s in recipe]
    p = tp.default_params(seed=1)
    out = tp.partition_batch(graphs, ks, 0.03, p, concurrency=8)
    for i, ((xadj, adj), g, (part, st)) in enumerate(zip(csr, graphs, out)):
        single, sst = tp.partition(g, ks[i], 0.03, p)
        want, wst = oracle.partition(oracle.Graph(xadj, adj), ks[i], 0.03, oracle.Params(seed=1))
        got = part.cpu().numpy()
        assert np.array_equal(got, single.cpu().numpy()), i
        assert np.array_equal(got, want), i
        assert st["cut"] == sst["cut"] == wst["cut"], i


def test_batch_independent_of_streams_and_knobs(small_batch):
    recipe, _, graphs = small_batch
    ks = [s["k"] for s in recipe]
    base = [p.cpu().numpy() for p, _ in tp.partition_batch(graphs, ks, 0.03, tp.default_params(),
                                                          concurrency=1)]
    for conc, knobs in ((3, {"tier_lane": 0, "tier_small": 32, "warps_per_block": 4}),
                        (32, {"tier_lane": 16, "tier_small": 64, "tier_mid": 256})):
        out = tp.partition_batch(graphs, ks, 0.03, tp.default_params(**knobs), concurrency=conc)
        for i, (part, _) in enumerate(out):
            assert np.array_equal(part.cpu().numpy(), base[i]), (conc, knobs, i)


def test_batch_rejects_bad_arguments(small_batch):
    _, _, graphs = small_batch
    with pytest.raises(tp.TpError):
        tp.partition_batch([graphs[0], graphs[0]], [2, 2], 0.03)  # same handle twice
    with pytest.raises(tp.TpError):
        tp.partition_batch(graphs[:2], [2, 0], 0.03)  # k < 1
    assert tp.partition_batch([], [], 0.03) == []


def test_autotune_picks_a_result_preserving_setting(small_batch):
    recipe, _, graphs = small_batch
    ks = [s["k"] for s in recipe]
    p, table = autotune.autotune(graphs[:12], ks[:12], sample=6, repeats=1)
    assert 1 <= len(table) <= 1 + len(list(autotune.candidates()))
    tuned = tp.partition_batch(graphs[:12], ks[:12], 0.03, p)
    plain = tp.partition_batch(graphs[:12], ks[:12], 0.03, tp.default_params(), concurrency=1)
    for (a, _), (b, _) in zip(tuned, plain):
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_compressed_graph_too_small_to_coarsen():
    # n <= c_lim * k: the initial partitioner sees the level-0 graph itself
    xadj, adj = synth.rhg(600, 16.0, 2.8, 9)
    z = tp.graph_from_csr(xadj, adj).compress()
    part, st = tp.partition(z, 8, 0.03, tp.default_params(seed=2))
    want, wst = oracle.partition(oracle.Graph(xadj, adj), 8, 0.03, oracle.Params(seed=2))
    assert st["levels"] == 1
    assert np.array_equal(part.cpu().numpy(), want) and st["cut"] == wst["cut"]


def _weighted(xadj, adj, seed):
    """Random vertex weights 1..40 and symmetric edge weights 1..500."""
    rng = np.random.default_rng(seed)
    n = len(xadj) - 1
    vw = rng.integers(1, 41, size=n).astype(np.int64)
    src = np.repeat(np.arange(n), np.diff(xadj))
    lo, hi = np.minimum(src, adj), np.maximum(src, adj)
    ew = (((lo * 2654435761 + hi * 40503) % 499) + 1).astype(np.int64)  # same for (u,v) and (v,u)
    return vw, ew


def _check_against_oracle(graphs, hosts, ks, p, op, conc=4):
    out = tp.partition_batch(graphs, ks, 0.03, p, concurrency=conc)
    for i, ((part, st), h) in enumerate(zip(out, hosts)):
        want, wst = oracle.partition(h, ks[i], 0.03, op)
        assert np.array_equal(part.cpu().numpy(), want), i
        for key in ("cut", "levels", "level_n", "level_m2", "max_block_weight", "l_max", "u_max",
                    "balanced"):
            assert st[key] == wst[key], (i, key, st[key], wst[key])


def test_batch_mixes_trivial_weighted_and_large_k_graphs():
    """k = 1, no vertices, weighted graphs next to unit ones, k above n / c_lim
    (no coarsening), and graphs that stop coarsening at different levels, all
    in one union."""
    specs = []
    xs = [synth.gnm(1500, 6000, 1), synth.rgg2d(2500, 12.0, 2), synth.rhg(2000, 16.0, 2.8, 3),
          synth.gnm(700, 2100, 4), synth.rgg2d(3000, 10.0, 5), synth.rhg(1200, 12.0, 2.6, 6)]
    ks = [4, 1, 8, 64, 2, 16]
    graphs, hosts = [], []
    for i, (xadj, adj) in enumerate(xs):
        if i in (2, 4):
            vw, ew = _weighted(xadj, adj, i)
            graphs.append(tp.graph_from_csr(xadj, adj, vw, ew))
            hosts.append(oracle.Graph(xadj, adj, vw, ew))
        else:
            graphs.append(tp.graph_from_csr(xadj, adj))
            hosts.append(oracle.Graph(xadj, adj))
    ex, ea = np.zeros(1, np.int64), np.zeros(0, np.int32)  # no vertices
    graphs.append(tp.graph_from_csr(ex, ea))
    hosts.append(oracle.Graph(ex, ea))
    ks.append(4)
    _check_against_oracle(graphs, hosts, ks, tp.default_params(seed=5), oracle.Params(seed=5))


def test_batch_with_graphs_that_stop_shrinking():
    """Without two-hop packing an edgeless graph does not shrink at all, so it
    leaves the union after its first clustering, while the others go on; a
    depth limit cuts the rest."""
    xadj_e = np.zeros(3001, np.int64)  # 3000 isolated vertices
    adj_e = np.zeros(0, np.int32)
    xs = [synth.rgg2d(4000, 12.0, 7), (xadj_e, adj_e), synth.gnm(3500, 14000, 8)]
    ks = [2, 2, 4]
    for max_levels in (64, 2):
        p = tp.default_params(seed=3, two_hop=0, max_levels=max_levels)
        op = oracle.Params(seed=3, two_hop=0, max_levels=max_levels)
        graphs = [tp.graph_from_csr(x, a) for x, a in xs]
        hosts = [oracle.Graph(x, a) for x, a in xs]
        _check_against_oracle(graphs, hosts, ks, p, op)


def test_batch_of_one_equals_single():
    xadj, adj = synth.rhg(3000, 16.0, 2.8, 11)
    g = tp.graph_from_csr(xadj, adj)
    (part, st), = tp.partition_batch([g], [8], 0.03, tp.default_params(seed=4))
    single, sst = tp.partition(g, 8, 0.03, tp.default_params(seed=4))
    assert np.array_equal(part.cpu().numpy(), single.cpu().numpy())
    assert st["cut"] == sst["cut"] and st["level_n"] == sst["level_n"]
