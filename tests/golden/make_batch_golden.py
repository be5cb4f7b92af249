#!/usr/bin/env python3
"""Writes the oracle's partitions of the batched workload to
tests/golden/batch4096.json.

The batched workload is synth.batch_recipe(4096, seed=1) (n log-uniform in
[2^8, 2^16], G(n,m) / RGG-2D / RHG in turn, k in {2,4,8,16,32}, eps = 0.03,
params seed 1). The oracle partitions all 4 096 graphs; the fixture stores
the SHA-256 of every partition concatenated in recipe order (int32 each), the
sum of the cuts, and for a sample (every 64th graph in order of n) the
graph's index, size, k, cut and partition SHA-256, so the GPU test can
compare the whole batch at benchmark size without running the oracle. Only
oracle/ and synth/ are used (about four minutes on one host core).

    python tests/golden/make_batch_golden.py
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
COUNT, SEED, EPS, STRIDE = 4096, 1, 0.03, 64


def sample_indices(recipe):
    order = sorted(range(len(recipe)), key=lambda i: (recipe[i]["n"], i))
    return sorted(order[j] for j in range(0, len(order), STRIDE))


def main():
    oracle.build()
    synth.build()
    recipe = synth.batch_recipe(COUNT, seed=SEED)
    sample = set(sample_indices(recipe))
    out = []
    whole = hashlib.sha256()
    cut_sum = 0
    t0 = time.time()
    for i, r in enumerate(recipe):
        xadj, adj = synth.batch_graph(r)
        part, st = oracle.partition(oracle.Graph(xadj, adj), r["k"], EPS, oracle.Params(seed=SEED))
        data = np.ascontiguousarray(part, np.int32).data
        whole.update(data)
        cut_sum += int(st["cut"])
        if i in sample:
            out.append({"index": i, "gen": r["gen"], "n": len(xadj) - 1, "m2": int(len(adj)),
                        "k": r["k"], "cut": int(st["cut"]), "levels": int(st["levels"]),
                        "partition_sha256": hashlib.sha256(data).hexdigest()})
        if i % 256 == 0:
            print(f"graph {i} ({time.time() - t0:.0f} s)", flush=True)
    rec = {"what": "oracle partitions of synth.batch_recipe(4096, seed=1), eps 0.03, params seed 1: "
                   "SHA-256 of all partitions (int32, recipe order), sum of cuts, and every 64th "
                   "graph by n in detail",
           "count": COUNT, "seed": SEED, "eps": EPS, "stride": STRIDE,
           "all_partitions_sha256": whole.hexdigest(), "sum_cut": cut_sum, "sample": out,
           "oracle_seconds": round(time.time() - t0, 1)}
    with open(os.path.join(HERE, "batch4096.json"), "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
