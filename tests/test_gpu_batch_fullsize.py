"""Batched mode at the benchmark's size: the 4 096-graph recipe partitioned in
one batch call (one union graph per level) equals the oracle's partition of
every graph. The oracle's results are stored by
tests/golden/make_batch_golden.py (oracle/ and synth/ only) in
tests/golden/batch4096.json: a SHA-256 over all partitions in recipe order,
the sum of the cuts, and 64 graphs spread over the size range in detail."""
import hashlib
import json
import os

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096.json")


def test_batch4096_equals_oracle():
    with open(GOLDEN) as f:
        gold = json.load(f)
    recipe = synth.batch_recipe(gold["count"], seed=gold["seed"])
    graphs = [tp.graph_from_csr(*synth.batch_graph(r)) for r in recipe]
    ks = [r["k"] for r in recipe]
    out = tp.partition_batch(graphs, ks, gold["eps"], tp.default_params(seed=gold["seed"]))
    parts = [np.ascontiguousarray(part.cpu().numpy(), np.int32) for part, _ in out]
    for s in gold["sample"]:
        i = s["index"]
        assert len(parts[i]) == s["n"], i
        assert hashlib.sha256(parts[i].data).hexdigest() == s["partition_sha256"], i
        assert out[i][1]["cut"] == s["cut"] and out[i][1]["levels"] == s["levels"], i
    assert sum(st["cut"] for _, st in out) == gold["sum_cut"]
    whole = hashlib.sha256()
    for p in parts:
        whole.update(p.data)
    assert whole.hexdigest() == gold["all_partitions_sha256"]
