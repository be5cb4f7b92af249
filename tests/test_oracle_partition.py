"""Pins for the oracle's balance caps, cut, projection, initial partitioning,
rebalancing, refinement and the multilevel driver (problem statement of the
paper's introduction; Sections "The Multilevel Scheme" and "KaMinPar")."""
import math
import os

import numpy as np
import pytest

import oracle
import synth
from tests import _brute as bf

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_caps_golden():
    with open(os.path.join(GOLD, "caps.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for W, k, eps_ppm, l_max, U in (map(int, r) for r in rows):
        assert oracle.block_cap(W, k, eps_ppm) == l_max
        assert oracle.cluster_cap(W, k, eps_ppm) == U
    assert oracle.eps_to_ppm(0.03) == 30000


@pytest.mark.parametrize("seed", range(5))
def test_cut_and_weights_bruteforce(seed):
    rng = np.random.default_rng(seed)
    xadj, adj, ew, vw = bf.random_graph(rng, 20, 0.3, 7)
    g = oracle.Graph(xadj, adj, vw, ew)
    part = rng.integers(0, 4, size=20).astype(np.int32)
    assert oracle.cut(g, part) == bf.cut(xadj, adj, ew, part)
    assert np.array_equal(oracle.block_weights(g, part, 4), np.bincount(part, weights=vw, minlength=4))


def test_projection_preserves_cut_and_weights():
    xadj, adj = synth.rgg2d(6000, 16.0, 9)
    g = oracle.Graph(xadj, adj)
    C = oracle.cluster(g, 30, oracle.Params(), 0)
    cg, mp = oracle.contract(g, C)
    rng = np.random.default_rng(1)
    coarse_part = rng.integers(0, 8, size=cg.n).astype(np.int32)
    fine_part = coarse_part[mp]
    assert oracle.cut(g, fine_part) == oracle.cut(cg, coarse_part)
    assert np.array_equal(oracle.block_weights(g, fine_part, 8), oracle.block_weights(cg, coarse_part, 8))


@pytest.mark.parametrize("seed", range(6))
def test_bisection_not_below_optimum(seed):
    rng = np.random.default_rng(50 + seed)
    xadj, adj, ew, vw = bf.random_graph(rng, 12, 0.35, 3)
    g = oracle.Graph(xadj, adj, vw, ew)
    W = int(vw.sum())
    l_max = oracle.block_cap(W, 2, 30000)
    part = oracle.initial_partition(g, 2, l_max, oracle.Params(seed=seed))
    B = oracle.block_weights(g, part, 2)
    assert set(np.unique(part)) <= {0, 1}
    opt = bf.min_bisection_cut(xadj, adj, ew, vw, l_max, l_max)
    if B.max() <= l_max and opt is not None:
        assert oracle.cut(g, part) >= opt


def test_two_disjoint_cliques_cut_zero():
    n = 40
    edges = [(u, v) for base in (0, 20) for u in range(base, base + 20) for v in range(u + 1, base + 20)]
    nb = [[] for _ in range(n)]
    for u, v in edges:
        nb[u].append(v)
        nb[v].append(u)
    xadj = np.zeros(n + 1, np.int64)
    adj = []
    for u in range(n):
        adj += sorted(nb[u])
        xadj[u + 1] = len(adj)
    g = oracle.Graph(xadj, np.array(adj, np.int32))
    part, st = oracle.partition(g, 2, 0.03, oracle.Params())
    assert st["cut"] == 0 and st["balanced"]


@pytest.mark.parametrize("seed", range(8))
def test_rebalance_by_enumeration(seed):
    rng = np.random.default_rng(200 + seed)
    xadj, adj, ew, vw = bf.random_graph(rng, 14, 0.3, 4)
    g = oracle.Graph(xadj, adj, vw, ew)
    k = 3
    part = np.zeros(14, np.int32)
    part[rng.random(14) < 0.2] = 1
    B = oracle.block_weights(g, part, k)
    l_max = int(vw.sum()) // k + 2
    want_part, want_B, want_r = bf.rebalance(xadj, adj, ew, vw, part, B, k, l_max)
    got_part, got_B = part.copy(), B.copy()
    r = oracle.rebalance(g, got_part, got_B, k, l_max)
    assert r == want_r
    assert list(got_part) == want_part and list(got_B) == want_B
    if r == 0:
        assert got_B.max() <= l_max


def test_refine_keeps_caps_and_does_not_raise_cut():
    xadj, adj = synth.rgg2d(8000, 16.0, 4)
    g = oracle.Graph(xadj, adj)
    k = 8
    rng = np.random.default_rng(3)
    part = (np.arange(g.n) * k // g.n).astype(np.int32)  # contiguous id ranges
    B = oracle.block_weights(g, part, k)
    l_max = oracle.block_cap(g.n, k, 30000)
    before = oracle.cut(g, part)
    oracle.refine(g, part, B, k, l_max, oracle.Params(), 0)
    assert np.array_equal(B, oracle.block_weights(g, part, k))
    assert B.max() <= l_max
    # refinement improves this deliberately poor start (contiguous id ranges)
    assert oracle.cut(g, part) <= before


@pytest.mark.parametrize("kind,k", [("gnm", 8), ("rgg", 16), ("rmat", 32)])
def test_partition_balanced_deterministic(kind, k):
    if kind == "gnm":
        xadj, adj = synth.gnm(1 << 13, 1 << 16, 1)
    elif kind == "rgg":
        xadj, adj = synth.rgg2d(1 << 14, 16.0, 1)
    else:
        xadj, adj = synth.rmat(13, 16, seed=1)
    g = oracle.Graph(xadj, adj)
    p = oracle.Params()
    part, st = oracle.partition(g, k, 0.03, p)
    assert part.min() >= 0 and part.max() < k
    assert st["balanced"] and st["max_block_weight"] <= st["l_max"]
    assert st["cut"] == oracle.cut(g, part)
    part2, st2 = oracle.partition(g, k, 0.03, p)
    assert np.array_equal(part, part2) and st == st2
    # the hierarchy shrinks by at least 5% per level
    ln = st["level_n"]
    assert all(20 * b <= 19 * a for a, b in zip(ln, ln[1:]))
    # a random partition of the same graph cuts more
    rnd = np.random.default_rng(0).integers(0, k, size=g.n).astype(np.int32)
    assert st["cut"] < oracle.cut(g, rnd)


def test_partition_k1_and_empty():
    xadj, adj = synth.gnm(100, 300, 1)
    g = oracle.Graph(xadj, adj)
    part, st = oracle.partition(g, 1, 0.03, oracle.Params())
    assert not part.any() and st["cut"] == 0
    g0 = oracle.Graph(np.zeros(1, np.int64), np.zeros(0, np.int32))
    part, st = oracle.partition(g0, 4, 0.03, oracle.Params())
    assert len(part) == 0 and st["cut"] == 0


def _bfs_growing_restated(xadj, adj, ew, vw, seed, attempts):
    """k = 2 without 2-way refinement, written out from the definition: per
    attempt a, FIFO breadth-first order from vertex round_key(seed, ip-seed,
    node key, a) mod n (neighbours in ascending id, unreached vertices
    appended in ascending id); side 0 is the longest prefix of that order of
    weight <= floor(W * 1 / 2); the attempt with the smallest cut wins (the
    lowest attempt on ties)."""
    from collections import deque

    n = len(xadj) - 1
    IPSEED = 0x495053656564566B  # "IPSeedVk"
    key = (0 << 32) | 2  # root node: block offset 0, two blocks
    W = int(np.sum(vw))
    target0 = (W * 1) // 2
    best = None
    for a in range(attempts):
        s0 = bf.round_key(seed, IPSEED, key, a) % n
        seen = [False] * n
        order = [s0]
        seen[s0] = True
        q = deque([s0])
        while q:
            u = q.popleft()
            for e in range(xadj[u], xadj[u + 1]):
                v = int(adj[e])
                if not seen[v]:
                    seen[v] = True
                    order.append(v)
                    q.append(v)
        order += [u for u in range(n) if not seen[u]]
        side = np.ones(n, np.int32)
        acc = 0
        for u in order:
            acc += int(vw[u])
            if acc > target0:
                break
            side[u] = 0
        c = bf.cut(xadj, adj, ew, side)
        if best is None or c < best[0]:
            best = (c, side)
    return best[1]


@pytest.mark.parametrize("seed", range(10))
def test_bfs_growing_bisection_by_restatement(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(5, 40))
    xadj, adj, ew, vw = bf.random_graph(rng, n, float(rng.uniform(0.05, 0.3)), max_w=3)
    W = int(np.sum(vw))
    l_max = W  # no cap binds: the growing step alone decides
    got = oracle.initial_partition(oracle.Graph(xadj, adj, vw=vw, ew=ew), 2, l_max,
                                   oracle.Params(seed=7, refine_rounds=0, ip_attempts=8))
    want = _bfs_growing_restated(xadj, adj, ew, vw, 7, 8)
    assert list(got) == list(want)


def _recursive_bisection_restated(xadj, adj, ew, vw, k, l_max, seed, attempts, rounds, S):
    """Initial partitioning written out from its definition: a tree node owns
    an ascending vertex list and the blocks [offset, offset + kk); with
    k0 = ceil(kk/2), k1 = floor(kk/2) it works on the induced subgraph in
    local ids, grows side 0 by BFS from a hashed seed up to floor(W k0 / kk)
    in every attempt, runs the 2-way LP (blocks {0, 1}, caps k0 L_max and
    k1 L_max, keys (seed, ip-lp, node key, (attempt << 8) + round)), keeps the
    smallest cut (lowest attempt on ties) and recurses into both sides."""
    from collections import deque

    IPSEED = int.from_bytes(b"IPSeedVk", "big")
    IPLP = int.from_bytes(b"IPLP2Way", "big")
    TIE = int.from_bytes(b"TieBrekr", "big")
    part = np.zeros(len(xadj) - 1, np.int32)

    def node(vs, kk, offset):
        if kk == 1:
            part[vs] = offset
            return
        ns = len(vs)
        if ns == 0:
            return
        k0, k1 = (kk + 1) // 2, kk // 2
        loc = {int(v): i for i, v in enumerate(vs)}
        sx, sa, se = [0], [], []
        for v in vs:
            for e in range(xadj[v], xadj[v + 1]):
                if int(adj[e]) in loc:
                    sa.append(loc[int(adj[e])])
                    se.append(int(ew[e]))
            sx.append(len(sa))
        sx, sa, se = np.array(sx, np.int64), np.array(sa, np.int32), np.array(se, np.int64)
        svw = np.array([int(vw[v]) for v in vs], np.int64)
        W = int(svw.sum())
        target0 = W * k0 // kk
        caps = np.array([k0 * l_max, k1 * l_max], np.int64)
        key = (offset << 32) | kk
        best = None
        for a in range(attempts):
            s0 = bf.round_key(seed, IPSEED, key, a) % ns
            seen = [False] * ns
            order, q = [s0], deque([s0])
            seen[s0] = True
            while q:
                x = q.popleft()
                for e in range(sx[x], sx[x + 1]):
                    y = int(sa[e])
                    if not seen[y]:
                        seen[y] = True
                        order.append(y)
                        q.append(y)
            order += [x for x in range(ns) if not seen[x]]
            side = np.ones(ns, np.int32)
            acc = 0
            for x in order:
                if acc + int(svw[x]) > target0:
                    break
                acc += int(svw[x])
                side[x] = 0
            lw = np.array([acc, W - acc], np.int64)
            for r in range(rounds):
                rk = bf.round_key(seed, IPLP, key, (a << 8) + r)
                for s in range(S):
                    side, lw = bf.subround(sx, sa, se, svw, side, lw, 2, caps, rk, S, s, TIE)
            c = bf.cut(sx, sa, se, side)
            if best is None or c < best[0]:
                best = (c, side.copy())
        side = best[1]
        node(vs[side == 0], k0, offset)
        node(vs[side == 1], k1, offset + k0)

    node(np.arange(len(xadj) - 1), k, 0)
    return part


def _ip_case(seed):
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(6, 30))
    xadj, adj, ew, vw = bf.random_graph(rng, n, float(rng.uniform(0.08, 0.35)), max_w=3)
    k = int(rng.integers(2, 7))
    W = int(np.sum(vw))
    l_max = -(-W // k) + int(rng.integers(0, 3))  # ceil(W/k) plus a little slack
    p = oracle.Params(seed=int(rng.integers(1, 2**40)), refine_rounds=int(rng.integers(0, 4)),
                      sub_rounds=int(rng.integers(1, 4)), ip_attempts=int(rng.integers(1, 5)))
    return xadj, adj, ew, vw, k, l_max, p


@pytest.mark.parametrize("seed", range(12))
def test_initial_partition_by_restatement(seed):
    xadj, adj, ew, vw, k, l_max, p = _ip_case(seed)
    got = oracle.initial_partition(oracle.Graph(xadj, adj, vw=vw, ew=ew), k, l_max, p)
    want = _recursive_bisection_restated(xadj, adj, ew, vw, k, l_max, p.seed, p.ip_attempts,
                                         p.refine_rounds, p.sub_rounds)
    assert list(got) == list(want)


def test_initial_partition_cases_exercise_lp():
    # the 2-way LP changes the grown sides in several of the cases above
    changed = 0
    for seed in range(12):
        xadj, adj, ew, vw, k, l_max, p = _ip_case(seed)
        a = _recursive_bisection_restated(xadj, adj, ew, vw, k, l_max, p.seed, p.ip_attempts,
                                          p.refine_rounds, p.sub_rounds)
        b = _recursive_bisection_restated(xadj, adj, ew, vw, k, l_max, p.seed, p.ip_attempts, 0,
                                          p.sub_rounds)
        changed += int(list(a) != list(b))
    assert changed >= 4, changed


def _multilevel_restated(xadj, adj, k, eps, p):
    """The multilevel driver written out from its definition, with the
    (separately pinned) oracle stages as steps: caps from integer ppm
    arithmetic; coarsen while n > c_lim k and fewer than max_levels graphs
    exist, discarding a level that keeps more than 95% of the vertices;
    initial partition of the coarsest graph; then from coarsest to finest:
    project, rebalance if some block exceeds L_max, refine (then FM, when
    asked for)."""
    g = oracle.Graph(xadj, adj)
    W = g.n
    ppm = int(math.floor(eps * 1e6 + 0.5))
    U = max(1, ppm * W // (10**6 * k))
    l_max = (10**6 + ppm) * (-(-W // k)) // 10**6
    levels, maps, level_n = [g], [], [g.n]
    if k > 1:
        while levels[-1].n > p.c_lim * k and len(levels) < min(p.max_levels, 64):
            fine = levels[-1]
            C = oracle.cluster(fine, U, p, len(levels) - 1)
            coarse, mp = oracle.contract(fine, C)
            if 20 * coarse.n > 19 * fine.n:
                break
            levels.append(coarse)
            maps.append(mp)
            level_n.append(coarse.n)
    L = len(levels) - 1
    cur = np.zeros(levels[L].n, np.int32)
    if k > 1:
        cur = oracle.initial_partition(levels[L], k, l_max, p).copy()
    for lv in range(L, -1, -1):
        if lv < L:
            cur = cur[maps[lv]].astype(np.int32)
        if k > 1:
            B = oracle.block_weights(levels[lv], cur, k)
            if B.max() > l_max:
                oracle.rebalance(levels[lv], cur, B, k, l_max)
            oracle.refine(levels[lv], cur, B, k, l_max, p, lv)
            if p.fm_passes > 0:
                oracle.fm_refine(levels[lv], cur, B, k, l_max, p.fm_passes)
    return cur, level_n, l_max


def _ml_cases():
    return [
        ("rgg", synth.rgg2d(3000, 12.0, 5), 4, 0.03, oracle.Params(seed=3, c_lim=20)),
        ("gnm", synth.gnm(2500, 9000, 6), 5, 0.0, oracle.Params(seed=4, c_lim=16)),
        ("rmat", synth.rmat(11, 8, seed=7), 8, 0.03, oracle.Params(seed=5, c_lim=10, two_hop=0)),
        ("rgg-2lv", synth.rgg2d(2000, 10.0, 8), 3, 0.1, oracle.Params(seed=6, c_lim=5,
                                                                      max_levels=2)),
        ("gnm-k1", synth.gnm(500, 2000, 9), 1, 0.03, oracle.Params(seed=7)),
        ("rgg-fm", synth.rgg2d(2500, 12.0, 6), 8, 0.03, oracle.Params(seed=8, c_lim=20,
                                                                     fm_passes=4)),
    ]


@pytest.mark.parametrize("case", range(6))
def test_multilevel_driver_by_restatement(case):
    name, (xadj, adj), k, eps, p = _ml_cases()[case]
    want, level_n, l_max = _multilevel_restated(xadj, adj, k, eps, p)
    got, st = oracle.partition(oracle.Graph(xadj, adj), k, eps, p)
    assert list(got) == list(want), name
    assert st["level_n"] == level_n and st["l_max"] == l_max, name


def test_stats_imbalance_and_block_weight():
    # W = 1000, k = 7: the perfectly balanced block weighs ceil(1000 / 7) = 143
    xadj, adj = synth.gnm(1000, 4000, 3)
    part, st = oracle.partition(oracle.Graph(xadj, adj), 7, 0.03, oracle.Params())
    B = np.bincount(part, minlength=7)
    assert st["max_block_weight"] == B.max()
    assert st["imbalance"] == B.max() / 143 - 1
    assert st["l_max"] == 147  # floor(1.03 * 143)


@pytest.mark.parametrize("gen", ["rgg", "rmat"])
def test_implicit_unit_weights_equal_explicit_arrays(gen):
    """A graph without weight arrays means unit weights: clustering,
    contraction, cut and the whole partition equal those of the same graph
    with explicit arrays of ones (large inputs are run without the arrays)."""
    xadj, adj = synth.rgg2d(3000, 12.0, 4) if gen == "rgg" else synth.rmat(11, 8, seed=4)
    ge = oracle.Graph(xadj, adj)
    gi = oracle.Graph(xadj, adj, implicit_unit=True)
    assert gi.vw is None and gi.ew is None
    p = oracle.Params(seed=3)
    Ce, Ci = oracle.cluster(ge, 20, p, 0), oracle.cluster(gi, 20, p, 0)
    assert np.array_equal(Ce, Ci)
    (ce, me), (ci, mi) = oracle.contract(ge, Ce), oracle.contract(gi, Ci)
    assert np.array_equal(me, mi) and np.array_equal(ce.adj, ci.adj) and np.array_equal(ce.ew, ci.ew)
    assert np.array_equal(ce.vw, ci.vw)
    for k in (2, 8, 13):
        pe, se = oracle.partition(ge, k, 0.03, p)
        pi, si = oracle.partition(gi, k, 0.03, p)
        assert np.array_equal(pe, pi) and se == si
        assert oracle.cut(gi, pi) == se["cut"]
    assert oracle.validate(gi) == 0
