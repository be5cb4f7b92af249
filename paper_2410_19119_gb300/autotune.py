"""Autotuner for the performance knobs of batched partitioning.

The knobs only decide which kernel rates a vertex and how work is laid out:
the degree bounds of the lane and warp tiers (tier_lane, tier_small,
tier_mid), the warps per block of the warp-per-vertex kernels
(warps_per_block) and the hash-table capacity of the warp tiers
(table_slack: slots per neighbour, so the table a vertex fills and scans has
the least power of two >= slack * degree slots). None of them changes a
result (integer sums commute and the rating order is total), so the tuner
may pick any of them by time alone.

A batch is partitioned as one union graph per level, so the tuner times
partition_batch on a sample that is itself a union spanning the batch's size
range (every stride-th graph in size order), and improves one knob at a time
from the defaults (coordinate descent, one pass): for each knob in turn it
tries every value with the others held, and keeps the fastest.
"""
import time

from . import default_params, partition_batch

KNOBS = (
    ("tier_lane", (0, 16, 32)),
    ("tier_small", (32, 64)),
    ("tier_mid", (128, 256, 512)),
    ("warps_per_block", (4, 8)),
    ("table_slack", (1, 2, 4)),
)


def candidates():
    """Every single-knob variation the tuner may try."""
    for name, values in KNOBS:
        for v in values:
            yield {name: v}


def sample_indices(graphs, size):
    """size graphs spread evenly over the batch sorted by n + 2m."""
    order = sorted(range(len(graphs)), key=lambda i: graphs[i].n + graphs[i].info()["m2"])
    if size >= len(order):
        return order
    step = len(order) / size
    return [order[int(j * step)] for j in range(size)]


def autotune(graphs, ks, eps=0.03, seed=1, sample=512, repeats=1):
    """Returns (params, table): the fastest knob set found on the sample and
    every (knobs, seconds) timed."""
    import torch

    idx = sample_indices(graphs, sample)
    gs, kk = [graphs[i] for i in idx], [ks[i] for i in idx]
    table = []
    seen = {}

    def timed(knobs):
        key = tuple(sorted(knobs.items()))
        if key in seen:
            return seen[key]
        p = default_params(seed=seed, **knobs)
        partition_batch(gs, kk, eps, p)  # warm-up (allocations, tier caches)
        dt = float("inf")
        for _ in range(repeats):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            partition_batch(gs, kk, eps, p)
            torch.cuda.synchronize()
            dt = min(dt, time.perf_counter() - t0)
        table.append((dict(knobs), dt))
        seen[key] = dt
        return dt

    d = default_params()
    best = {name: getattr(d, name) for name, _ in KNOBS}
    best_t = timed(best)
    for name, values in KNOBS:
        for v in values:
            trial = dict(best, **{name: v})
            t = timed(trial)
            if t < best_t:
                best, best_t = trial, t
    return default_params(seed=seed, **best), table
