#!/usr/bin/env python3
"""Writes the oracle's result for an R-MAT partition to tests/golden/.

The oracle (one host thread) partitions R-MAT scale S, edge factor 16,
(a,b,c,d) = (0.57, 0.19, 0.19, 0.05), symmetrised, deduplicated, self-loops
removed, unit weights, with k blocks, eps = 0.03 and seed 1, and also clusters
level 0 alone. The fixture stores a hash of the input graph, the parameters,
and the SHA-256 of the level-0 clustering and of the final partition with
every statistic, so that the GPU test can compare a full-size run without
running the oracle again. Only oracle/ and synth/ are used.

    python tests/golden/make_rmat_golden.py --scale 26 --k 256

takes about an hour and up to ~50 GB of host memory at scale 26.
"""
import argparse
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
EPS = 0.03


def graph_hash(xadj, adj):
    h = hashlib.sha256()
    h.update(np.ascontiguousarray(xadj, np.int64).data)
    h.update(np.ascontiguousarray(adj, np.int32).data)
    return h.hexdigest()


def array_hash(a):
    return hashlib.sha256(np.ascontiguousarray(a, np.int32).data).hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=26)
    ap.add_argument("--k", type=int, default=256)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    out = args.out or os.path.join(HERE, f"rmat{args.scale}_k{args.k}.json")
    oracle.build()
    synth.build()
    t0 = time.time()
    xadj, adj = synth.rmat(args.scale, 16, seed=args.seed)
    t_gen = time.time() - t0
    n, m2 = len(xadj) - 1, len(adj)
    print(f"generated n={n} m2={m2} in {t_gen:.0f} s", flush=True)
    g = oracle.Graph(xadj, adj, implicit_unit=True)
    p = oracle.Params(seed=args.seed)
    U = oracle.cluster_cap(n, args.k, oracle.eps_to_ppm(EPS))
    t0 = time.time()
    C = oracle.cluster(g, U, p, 0)
    t_cluster = time.time() - t0
    c_hash = array_hash(C)
    n_clusters = int(np.unique(C).size)
    del C
    print(f"level-0 clustering in {t_cluster:.0f} s: {n_clusters} clusters", flush=True)
    t0 = time.time()
    part, st = oracle.partition(g, args.k, EPS, p)
    t_part = time.time() - t0
    print(f"partition in {t_part:.0f} s: cut {st['cut']}", flush=True)
    B = np.bincount(part, minlength=args.k).astype(np.int64)
    rec = {
        "what": f"oracle partition of R-MAT scale {args.scale}, edge factor 16, "
                f"(0.57,0.19,0.19,0.05), symmetrised, deduplicated, self-loops removed, "
                f"unit weights",
        "generator": {"scale": args.scale, "edge_factor": 16, "a": 0.57, "b": 0.19, "c": 0.19,
                      "seed": args.seed},
        "graph_sha256": graph_hash(xadj, adj), "n": n, "m2": m2,
        "params": {"k": args.k, "eps": EPS, "seed": p.seed, "cluster_rounds": p.cluster_rounds,
                   "refine_rounds": p.refine_rounds, "sub_rounds": p.sub_rounds,
                   "c_lim": p.c_lim, "ip_attempts": p.ip_attempts, "two_hop": p.two_hop,
                   "max_levels": p.max_levels},
        "cluster_cap": U,
        "level0_clustering_sha256": c_hash, "level0_clusters": n_clusters,
        "partition_sha256": array_hash(part),
        "block_weights_sha256": hashlib.sha256(B.tobytes()).hexdigest(),
        "stats": {k: (v if not isinstance(v, (np.integer, np.floating)) else v.item())
                  for k, v in st.items()},
        "oracle_seconds": {"generate": round(t_gen, 1), "cluster_level0": round(t_cluster, 1),
                           "partition": round(t_part, 1)},
    }
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
        f.write("\n")
    print(f"wrote {out}", flush=True)


if __name__ == "__main__":
    main()
