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
    p, conc, table = autotune.autotune(graphs[:12], ks[:12], sample=6, repeats=1,
                                       concurrency=(2, 4))
    assert conc in (2, 4) and len(table) == 2 + len(list(autotune.candidates()))
    tuned = tp.partition_batch(graphs[:12], ks[:12], 0.03, p, concurrency=conc)
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
