"""Multi-rank host logic on the CPU (two gloo ranks): independent work units
are sharded over ranks with no collective on the data path, every unit's
result is the one a single process computes, and timings reduce to the
slowest rank. The GPU path runs one replica per rank the same way."""
import os
import socket

import numpy as np
import pytest

import bench
import oracle
import synth

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, recipe, out_q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws))
    import torch.distributed as d

    d.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        mine = bench.shard(len(recipe), rank, ws)
        results = {}
        for i in mine:
            xadj, adj = synth.batch_graph(recipe[i])
            part, st = oracle.partition(oracle.Graph(xadj, adj), recipe[i]["k"], 0.03,
                                        oracle.Params(seed=1))
            results[i] = (part.tolist(), st["cut"])
        gathered = [None] * ws
        d.all_gather_object(gathered, results)  # test only: collect the shards
        slowest = bench.max_over_ranks([10.0 * (rank + 1), -float(rank)], d)
        if rank == 0:
            merged = {}
            for g in gathered:
                merged.update(g)
            out_q.put((merged, slowest))
    finally:
        d.destroy_process_group()


def test_sharded_units_equal_single_process():
    recipe = synth.batch_recipe(10, seed=5, log2_lo=8.0, log2_hi=10.0)
    ws = 2
    assert sorted(sum((bench.shard(len(recipe), r, ws) for r in range(ws)), [])) == list(
        range(len(recipe)))
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, recipe, q)) for r in range(ws)]
    for p in procs:
        p.start()
    merged, slowest = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert slowest == [20.0, 0.0]  # element-wise max over the two ranks
    assert sorted(merged) == list(range(len(recipe)))
    for i, spec in enumerate(recipe):
        xadj, adj = synth.batch_graph(spec)
        part, st = oracle.partition(oracle.Graph(xadj, adj), spec["k"], 0.03, oracle.Params(seed=1))
        assert merged[i][0] == part.tolist() and merged[i][1] == st["cut"], i


def test_helpers_without_a_process_group():
    assert bench.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]
    assert bench.shard(5, 0, 1) == [0, 1, 2, 3, 4]
    assert bench.shard(5, 1, 2) == [1, 3]


def test_autotune_candidates_and_sample():
    from paper_2410_19119_gb300 import autotune

    cands = list(autotune.candidates())
    keys = {tuple(sorted(c.items())) for c in cands}
    assert len(keys) == len(cands) == sum(len(v) for _, v in autotune.KNOBS)
    assert all(c.get("tier_mid", 0) <= 512 for c in cands)  # the mid table holds degree <= 512
    assert {v for c in cands for k, v in c.items() if k == "table_slack"} <= {1, 2, 4, 8}
    import paper_2410_19119_gb300 as tp
    fields = {f for f, _ in tp._lib.Params._fields_}
    assert all(k in fields for c in cands for k in c)  # every knob is a tp_params field

    class G:
        def __init__(self, n, m2):
            self.n, self._m2 = n, m2

        def info(self):
            return {"m2": self._m2}

    gs = [G(n, 8 * n) for n in (5, 900, 30, 7000, 400, 12, 65000, 2000)]
    idx = autotune.sample_indices(gs, 4)
    assert len(idx) == 4 and len(set(idx)) == 4
    sizes = sorted(gs[i].n for i in idx)
    assert sizes[0] == 5 and sizes[-1] >= 2000  # spread from the smallest upwards
    assert sorted(autotune.sample_indices(gs, 99)) == list(range(len(gs)))


def test_autotune_coordinate_descent_picks_the_fastest_knobs(monkeypatch):
    """With a stubbed batch call whose cost depends on the knobs and a fake
    clock, the tuner improves one knob at a time from the defaults and keeps
    every improvement."""
    import types

    import torch

    from paper_2410_19119_gb300 import autotune

    clock = {"t": 0.0}
    best = {"tier_lane": 16, "tier_small": 64, "tier_mid": 256, "warps_per_block": 4,
            "table_slack": 1}

    def cost(p):
        return 1.0 + sum(0.1 for k, v in best.items() if getattr(p, k) != v)

    def fake_batch(gs, kk, eps, p, concurrency=1):
        clock["t"] += cost(p)

    monkeypatch.setattr(autotune, "partition_batch", fake_batch)
    monkeypatch.setattr(autotune, "time", types.SimpleNamespace(perf_counter=lambda: clock["t"]))
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)

    class G:
        def __init__(self, n):
            self.n = n

        def info(self):
            return {"m2": 8 * self.n}

    gs = [G(100 * (i + 1)) for i in range(20)]
    p, table = autotune.autotune(gs, [2] * 20, sample=5, repeats=1)
    assert {k: getattr(p, k) for k in best} == best
    assert abs(min(t for _, t in table) - 1.0) < 1e-9
    # the defaults first, then each knob's values with the others held
    assert len(table) <= 1 + sum(len(v) for _, v in autotune.KNOBS)
