"""The stored oracle results of the batched workload (tests/golden/batch4096.json)
still match the oracle: the smallest sampled graphs are partitioned again here
and compared with their stored hashes and cuts."""
import hashlib
import json
import os

import numpy as np

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch4096.json")


def test_stored_batch_results_match_the_oracle():
    with open(GOLDEN) as f:
        gold = json.load(f)
    recipe = synth.batch_recipe(gold["count"], seed=gold["seed"])
    small = sorted(gold["sample"], key=lambda s: s["n"])[:8]
    for s in small:
        r = recipe[s["index"]]
        xadj, adj = synth.batch_graph(r)
        assert (len(xadj) - 1, len(adj), r["k"]) == (s["n"], s["m2"], s["k"])
        part, st = oracle.partition(oracle.Graph(xadj, adj), r["k"], gold["eps"],
                                    oracle.Params(seed=gold["seed"]))
        assert hashlib.sha256(np.ascontiguousarray(part, np.int32).data).hexdigest() == \
            s["partition_sha256"], s["index"]
        assert st["cut"] == s["cut"] and st["levels"] == s["levels"]
