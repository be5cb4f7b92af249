"""The synchronous LP sub-round sharded over two gloo ranks on the CPU, as the
paper's distributed variant splits a graph (Section "KaMinPar": the
distributed partitioner runs label propagation on a 1-D vertex partition
with ghost vertices): each rank owns a vertex range and a set of labels
(clustering: the labels named after its vertices; refinement: blocks dealt
round robin). One sub-round is
  1. exchange labels and label weights (the snapshot, ghosts included);
  2. rate the owned active vertices against it;
  3. send each mover record to the owner of its target label;
  4. the owner approves per target (longest fitting prefix by gain desc,
     vertex asc) — owner-local, so no further agreement is needed;
  5. send the approvals back; apply them to owned vertices and owned labels.
The result equals the single-process sub-rounds exactly. This checks the
protocol on the host only: no GPU path shards one graph (each box here has
one GPU); the bench runs independent replicas instead."""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    xadj, adj = synth.rgg2d(2000, 10.0, 11)
    vw = np.random.default_rng(3).integers(1, 4, len(xadj) - 1).astype(np.int64)
    return xadj, adj, vw, 12, 3, 8, 77  # graph, node weights, cap, rounds, S, seed


def _gather(d, ws, obj):
    out = [None] * ws
    d.all_gather_object(out, obj)
    return out


def _refine_start(n, k):
    return np.random.default_rng(9).integers(0, k, n).astype(np.int32)


def _rank_main(rank, ws, port, out_q, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import torch.distributed as d

    d.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        xadj, adj, vw, cap, rounds, S, seed = _case()
        n = len(xadj) - 1
        g = oracle.Graph(xadj, adj, vw=vw)
        bounds = [n * r // ws for r in range(ws + 1)]
        lo, hi = bounds[rank], bounds[rank + 1]
        if mode == "cluster":  # labels are vertex ids, owned with their vertex
            nlabels = n
            label_own = np.arange(lo, hi, dtype=np.int32)
            lw_all = vw.copy()
            tag = oracle.tag(oracle.TAG_CLUSTER)
        else:  # refinement: labels are the K blocks, block b owned by rank b mod ws
            nlabels = K_BLOCKS
            part = _refine_start(n, K_BLOCKS)
            label_own = part[lo:hi].copy()
            lw_all = np.bincount(part, weights=vw, minlength=K_BLOCKS).astype(np.int64)
            cap = int(lw_all.max()) + 4
            tag = oracle.tag(oracle.TAG_REFINE)

        def owner(x):
            if mode == "cluster":
                return int(np.searchsorted(bounds, x, side="right") - 1)
            return x % ws

        mine = [x for x in range(nlabels) if owner(x) == rank]
        lw_own = {x: int(lw_all[x]) for x in mine}  # weights of the labels this rank owns
        for r in range(rounds):
            rk = oracle.round_key(seed, tag, 0, r)
            for s in range(S):
                # 1. snapshot: every rank's labels and label weights
                labels = np.concatenate(_gather(d, ws, label_own)).astype(np.int32)
                lw = np.zeros(nlabels, np.int64)
                for part_w in _gather(d, ws, lw_own):
                    for x, w in part_w.items():
                        lw[x] = w
                # 2. rate the owned active vertices
                moves = []
                for u in range(lo, hi):
                    hu, hv = oracle.vertex_hashes(rk, u)
                    if hu % S != s:
                        continue
                    moved, t, gain = oracle.rate_vertex_sorted(g, u, labels, lw, cap, hv=hv)
                    if moved:
                        moves.append((t, -gain, u, int(vw[u]), int(labels[u])))
                # 3. route the records to the owners of their targets
                routed = [m for part in _gather(d, ws, moves) for m in part if owner(m[0]) == rank]
                # 4. approval by the target's owner
                approved = []
                for t in sorted({m[0] for m in routed}):
                    mv = sorted(m for m in routed if m[0] == t)  # gain desc, then vertex asc
                    p = 0
                    for m in mv:
                        p += m[3]
                        if lw[t] + p <= cap:
                            approved.append(m)
                # 5. approvals back to everyone; apply to what this rank owns
                for t, _, u, w, src in (m for part in _gather(d, ws, approved) for m in part):
                    if lo <= u < hi:
                        label_own[u - lo] = t
                    if owner(t) == rank:
                        lw_own[t] += w
                    if owner(src) == rank:
                        lw_own[src] -= w
        result = _gather(d, ws, (label_own.tolist(), lw_own))
        if rank == 0:
            out_q.put(result)
    finally:
        d.destroy_process_group()


K_BLOCKS = 5


@pytest.mark.parametrize("mode", ["cluster", "refine"])
def test_sharded_subrounds_equal_single_process(mode):
    ws = 2
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q, mode)) for r in range(ws)]
    for p in procs:
        p.start()
    try:
        result = q.get(timeout=300)
    finally:
        for p in procs:
            p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    labels = np.concatenate([np.array(r[0], np.int32) for r in result])
    xadj, adj, vw, cap, rounds, S, seed = _case()
    n = len(xadj) - 1
    if mode == "cluster":
        nlabels, start, tag = n, np.arange(n, dtype=np.int32), oracle.TAG_CLUSTER
        want_w = vw.copy()
    else:
        nlabels, start, tag = K_BLOCKS, _refine_start(n, K_BLOCKS), oracle.TAG_REFINE
        want_w = np.bincount(start, weights=vw, minlength=K_BLOCKS).astype(np.int64)
        cap = int(want_w.max()) + 4
    lws = np.zeros(nlabels, np.int64)
    for r in result:
        for x, w in r[1].items():
            lws[x] = w
    want = start.copy()
    oracle.lp_rounds(oracle.Graph(xadj, adj, vw=vw), want, want_w, nlabels, cap, None, seed,
                     oracle.tag(tag), 0, 0, rounds, S)
    assert np.array_equal(labels, want) and np.array_equal(lws, want_w)
    assert np.count_nonzero(want != start) > n // 10  # the rounds did move vertices
