"""Pins for the oracle's k-way FM over the gain table: the search restated by
brute force (affinities recounted for every candidate, no gain table) on tiny
weighted graphs, and the invariants any correct FM keeps on larger graphs:
the cut drops by exactly the reported gain and never rises, block caps hold,
and when FM stops on a pass without gain no admissible move gains anything."""
import numpy as np
import pytest

import oracle
import synth
from tests import _brute as bf


def _aff(xadj, adj, ew, part, v, b):
    return sum(int(ew[e]) for e in range(xadj[v], xadj[v + 1]) if part[adj[e]] == b)


def _fm_restated(xadj, adj, ew, vw, part, B, k, l_max, passes):
    """The FM passes from their definition: best admissible move to a block
    holding a neighbour (gain desc, vertex asc, block asc) among unlocked
    vertices, until none is left; keep the shortest best-gain prefix; repeat
    while a pass gains."""
    n = len(xadj) - 1
    part, B = part.copy(), B.copy()
    total = 0
    for _ in range(passes):
        locked = [False] * n
        log, run, best, best_len = [], 0, 0, 0
        while True:
            cands = []
            for v in range(n):
                if locked[v]:
                    continue
                own = int(part[v])
                for t in sorted({int(part[adj[e]]) for e in range(xadj[v], xadj[v + 1])}):
                    if t == own or B[t] + vw[v] > l_max:
                        continue
                    g = _aff(xadj, adj, ew, part, v, t) - _aff(xadj, adj, ew, part, v, own)
                    cands.append((-g, v, t, g))
            if not cands:
                break
            _, v, t, g = min(cands)
            log.append((v, int(part[v]), t))
            B[part[v]] -= vw[v]
            B[t] += vw[v]
            part[v] = t
            locked[v] = True
            run += g
            if run > best:
                best, best_len = run, len(log)
        for v, frm, to in reversed(log[best_len:]):
            B[to] -= vw[v]
            B[frm] += vw[v]
            part[v] = frm
        total += best
        if best <= 0:
            break
    return part, B, total


def _tiny(seed):
    rng = np.random.default_rng(1200 + seed)
    n = int(rng.integers(6, 16))
    xadj, adj, ew, vw = bf.random_graph(rng, n, float(rng.uniform(0.2, 0.6)), max_w=5)
    k = int(rng.integers(2, 5))
    part = rng.integers(0, k, n).astype(np.int32)
    B = np.bincount(part, weights=vw, minlength=k).astype(np.int64)
    l_max = int(B.max()) + int(rng.integers(0, 6))
    return xadj, adj, ew, vw, k, part, B, l_max


@pytest.mark.parametrize("seed", range(16))
def test_fm_by_restatement(seed):
    xadj, adj, ew, vw, k, part, B, l_max = _tiny(seed)
    want_p, want_B, want_gain = _fm_restated(xadj, adj, ew, vw, part, B, k, l_max, 4)
    got_p, got_B = part.copy(), B.copy()
    gain = oracle.fm_refine(oracle.Graph(xadj, adj, vw=vw, ew=ew), got_p, got_B, k, l_max, 4)
    assert list(got_p) == list(want_p) and list(got_B) == list(want_B) and gain == want_gain


def test_fm_cases_improve_cuts():
    improved = 0
    for seed in range(16):
        xadj, adj, ew, vw, k, part, B, l_max = _tiny(seed)
        _, _, gain = _fm_restated(xadj, adj, ew, vw, part, B, k, l_max, 4)
        improved += gain > 0
    assert improved >= 10, improved


@pytest.mark.parametrize("kind,k", [("rgg", 4), ("gnm", 8), ("rmat", 16)])
def test_fm_invariants(kind, k):
    if kind == "rgg":
        xadj, adj = synth.rgg2d(1500, 10.0, 3)
    elif kind == "gnm":
        xadj, adj = synth.gnm(1200, 5000, 4)
    else:
        xadj, adj = synth.rmat(10, 8, seed=5)
    g = oracle.Graph(xadj, adj)
    n = g.n
    rng = np.random.default_rng(7)
    part = rng.integers(0, k, n).astype(np.int32)
    B = oracle.block_weights(g, part, k)
    l_max = oracle.block_cap(n, k, 30000)
    if B.max() > l_max:
        oracle.rebalance(g, part, B, k, l_max)
    before = oracle.cut(g, part)
    gain = oracle.fm_refine(g, part, B, k, l_max, 50)
    after = oracle.cut(g, part)
    assert gain >= 0 and after == before - gain and gain > 0
    assert np.array_equal(B, oracle.block_weights(g, part, k)) and B.max() <= l_max
    # FM stopped on a pass without gain (50 passes is ample here): no
    # admissible move to a neighbouring block has a positive gain
    t = oracle.GainTable(g, part, k)
    for v in range(n):
        own = int(part[v])
        for e in range(xadj[v], xadj[v + 1]):
            x = int(part[adj[e]])
            if x != own and B[x] + 1 <= l_max:
                assert t.get(v, x) - t.get(v, own) <= 0, (v, x)


def test_fm_hand_case_target_ties():
    # path 1 - 0 - 2 in blocks [0, 1, 2], unit weights, L_max = 3. Pass 1:
    # every admissible move gains 1; the smallest vertex 0 goes to the smaller
    # of its two equal blocks, 1. Then only vertex 2 can move (to block 1,
    # gain 1). Pass 2 has no admissible move. Result [1, 1, 1], gain 2.
    xadj = np.array([0, 2, 3, 4], np.int64)
    adj = np.array([1, 2, 0, 0], np.int32)
    part = np.array([0, 1, 2], np.int32)
    B = np.ones(3, np.int64)
    gain = oracle.fm_refine(oracle.Graph(xadj, adj), part, B, 3, 3, 4)
    assert list(part) == [1, 1, 1] and list(B) == [0, 3, 0] and gain == 2
