"""Pins for the oracle's hashing and label propagation (Algorithm 1 made
synchronous; size constraint; two-hop packing)."""
import numpy as np
import pytest

import oracle
import synth
from tests import _brute as bf

# splitmix64 started from state 0 (published reference outputs of the
# generator of Steele, Lea and Flood): outputs are mix64(i * gamma), i = 1, 2, 3.
SPLITMIX64_FROM_ZERO = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_mix64_published_vectors():
    g = bf.GAMMA
    for i, want in enumerate(SPLITMIX64_FROM_ZERO, start=1):
        assert oracle.mix64((i * g) & bf.M64) == want
    # step(h, x) absorbs x + gamma: from h = 0 it is the first output
    assert oracle.step(0, 0) == SPLITMIX64_FROM_ZERO[0]
    assert oracle.step(0, g) == SPLITMIX64_FROM_ZERO[1]


def test_hash_agrees_with_bruteforce():
    rng = np.random.default_rng(0)
    for _ in range(200):
        a, b, c, d = (int(x) for x in rng.integers(0, 2**63, 4))
        assert oracle.round_key(a, b, c, d) == bf.round_key(a, b, c, d)
    tags = {oracle.tag(i) for i in range(6)}
    assert len(tags) == 6 and 0 not in tags


def _tiny(seed, n=10, p=0.35, max_w=3):
    rng = np.random.default_rng(seed)
    xadj, adj, ew, vw = bf.random_graph(rng, n, p, max_w)
    return rng, xadj, adj, ew, vw


@pytest.mark.parametrize("seed", range(12))
def test_rating_argmax_by_enumeration(seed):
    rng, xadj, adj, ew, vw = _tiny(seed)
    n = len(xadj) - 1
    g = oracle.Graph(xadj, adj, vw, ew)
    nlabels = n
    label = rng.integers(0, nlabels, size=n).astype(np.int32)
    lw = np.zeros(nlabels, np.int64)
    np.add.at(lw, label, vw)
    cap = rng.integers(1, 12, size=nlabels).astype(np.int64)
    for u in range(n):
        for ignore in (False, True):
            hv = int(rng.integers(0, 2**63))
            want = bf.rate(xadj, adj, ew, vw, u, label, lw, nlabels, cap, ignore, hv)
            for rate in (oracle.rate_vertex, oracle.rate_vertex_sorted):
                got = rate(g, u, label, lw, 0, cap, ignore, hv)
                assert got[0] == want[0], (u, got, want)
                if want[0]:
                    assert got[1:] == want[1:], (u, got, want)


@pytest.mark.parametrize("seed", range(16))
def test_subround_by_enumeration(seed):
    rng, xadj, adj, ew, vw = _tiny(100 + seed, n=12, p=0.4, max_w=4)
    n = len(xadj) - 1
    g = oracle.Graph(xadj, adj, vw, ew)
    S = int(rng.integers(1, 4))
    nlabels = n
    label = np.arange(n, dtype=np.int32)
    lw = vw.copy()
    capv = int(rng.integers(1, 10))
    cap = np.full(nlabels, capv, np.int64)
    for r in range(3):
        rk = int(rng.integers(0, 2**63))
        for s in range(S):
            want_l, want_w = bf.subround(xadj, adj, ew, vw, label, lw, nlabels, cap, rk, S, s,
                                         oracle.tag(oracle.TAG_TIE))
            oracle.lp_subround(g, label, lw, nlabels, capv, None, rk, S, s)
            assert np.array_equal(label, want_l) and np.array_equal(lw, want_w)


@pytest.mark.parametrize("kind", ["gnm", "rgg", "rmat"])
def test_cluster_cap_invariant(kind):
    if kind == "gnm":
        xadj, adj = synth.gnm(4000, 30000, 1)
    elif kind == "rgg":
        xadj, adj = synth.rgg2d(4000, 16.0, 1)
    else:
        xadj, adj = synth.rmat(12, 16, seed=1)
    g = oracle.Graph(xadj, adj)
    n = g.n
    U = 25
    p = oracle.Params(two_hop=0)
    label = np.arange(n, dtype=np.int32)
    lw = np.ones(n, np.int64)
    for r in range(5):
        rk = oracle.round_key(1, oracle.tag(oracle.TAG_CLUSTER), 0, r)
        for s in range(8):
            oracle.lp_subround(g, label, lw, n, U, None, rk, 8, s)
            recount = np.bincount(label, minlength=n)
            assert np.array_equal(recount, lw)
            assert lw.max() <= U and lw.sum() == n
    C = oracle.cluster(g, U, oracle.Params(), 0)
    sizes = np.bincount(C, minlength=n)
    assert sizes.max() <= U and sizes.sum() == n


def test_first_round_moves_every_nonisolated_vertex_possible():
    # a path 0-1-2-3: in round 0 every active vertex sees only singletons with
    # rating 1 > 0 = R[own], so it moves unless its target is full
    xadj = np.array([0, 1, 3, 5, 6], np.int64)
    adj = np.array([1, 0, 2, 1, 3, 2], np.int32)
    g = oracle.Graph(xadj, adj)
    label = np.arange(4, dtype=np.int32)
    lw = np.ones(4, np.int64)
    moved = oracle.lp_subround(g, label, lw, 4, 10, None, 12345, 1, 0)
    assert moved == 4  # S = 1: all active, all move (to a neighbour's label)
    assert all(label[u] in (u - 1, u + 1) for u in range(4))


def test_two_hop_isolated_packing():
    # 10 isolated vertices, U = 4: bins of P//4 -> {0..3}, {4..7}, {8, 9}
    n = 10
    g = oracle.Graph(np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
    C = np.arange(n, dtype=np.int32)
    Wc = np.ones(n, np.int64)
    oracle.two_hop(g, C, Wc, 4, 1, 0)
    assert list(C) == [0, 0, 0, 0, 4, 4, 4, 4, 8, 8]


def test_two_hop_straddler_stays_alone():
    # isolated vertices of weights 3,3,3,3 and U = 7: prefixes 0,3,6,9 ->
    # bins 0,0,0(straddles 6+3>7),1 -> groups {0,1}, {2} alone, {3}
    n = 4
    g = oracle.Graph(np.zeros(n + 1, np.int64), np.zeros(0, np.int32), vw=np.full(n, 3))
    C = np.arange(n, dtype=np.int32)
    Wc = np.full(n, 3, np.int64)
    oracle.two_hop(g, C, Wc, 7, 1, 0)
    assert list(C) == [0, 0, 2, 3]


def test_two_hop_shared_favourite():
    # star: centre 0 with leaves 1..9. The centre's cluster {0,1,2} is full
    # (U = 3); leaves 3..9 are singletons whose favourite is cluster 0 and get
    # packed three by three in id order.
    n = 10
    xadj = np.zeros(n + 1, np.int64)
    adj = []
    nb = {0: list(range(1, n))}
    for v in range(1, n):
        nb[v] = [0]
    for u in range(n):
        adj += nb[u]
        xadj[u + 1] = len(adj)
    g = oracle.Graph(xadj, np.array(adj, np.int32))
    C = np.array([0, 0, 0, 3, 4, 5, 6, 7, 8, 9], np.int32)
    Wc = np.zeros(n, np.int64)
    np.add.at(Wc, C, 1)
    oracle.two_hop(g, C, Wc, 3, 1, 0)
    assert list(C) == [0, 0, 0, 3, 3, 3, 6, 6, 6, 9]


def _two_hop_restated(xadj, adj, ew, vw, C, Wc, U, seed, level):
    """Two-hop packing written out from its definition: singletons (C[u] = u
    and Wc[u] = c(u)) keyed by their favourite cluster (best rating ignoring
    the cap; n if none), sorted by (key, u); inside a key, exclusive weight
    prefix P puts u in bin P // U unless it straddles the bin's end (then it
    stays alone); every bin becomes one cluster named after its first member."""
    n = len(xadj) - 1
    TWOHOP, TIE = 0x54776F486F704D74, 0x5469654272656B72  # tags "TwoHopMt", "TieBrekr"
    rk = bf.round_key(seed, TWOHOP, level, 0)
    single = [u for u in range(n) if C[u] == u and Wc[u] == vw[u]]
    keyed = []
    for u in single:
        hv = bf.step(bf.step(rk, u), TIE)
        ok, t, _ = bf.rate(xadj, adj, ew, vw, u, C, Wc, n, None, True, hv)
        keyed.append((t if ok else n, u))
    keyed.sort()
    out = C.copy()
    i = 0
    while i < len(keyed):
        j = i
        while j < len(keyed) and keyed[j][0] == keyed[i][0]:
            j += 1
        P, first = 0, {}
        for _, u in keyed[i:j]:
            b = P // U
            if P + vw[u] <= (b + 1) * U:
                first.setdefault(b, u)
                out[u] = first[b]
            P += vw[u]
        i = j
    return out


def _two_hop_case(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(8, 21))
    xadj, adj, ew, vw = bf.random_graph(rng, n, float(rng.uniform(0.05, 0.35)), max_w=3)
    reps = [u for u in range(n) if rng.random() < 0.8]
    C = np.arange(n, dtype=np.int32)
    for u in range(n):  # some vertices already joined another representative
        if u not in reps and reps and rng.random() < 0.5:
            C[u] = reps[int(rng.integers(len(reps)))]
    Wc = np.zeros(n, np.int64)
    np.add.at(Wc, C, vw)
    return xadj, adj, ew, vw, C, Wc, int(rng.integers(3, 11))


def test_two_hop_cases_exercise_packing():
    moved = [int(np.sum(_two_hop_restated(*_two_hop_case(s), 5, 2) != _two_hop_case(s)[4]))
             for s in range(12)]
    assert sum(m > 0 for m in moved) >= 8 and sum(moved) >= 20


@pytest.mark.parametrize("seed", range(12))
def test_two_hop_by_restatement(seed):
    xadj, adj, ew, vw, C, Wc, U = _two_hop_case(seed)
    want = _two_hop_restated(xadj, adj, ew, vw, C, Wc, U, 5, 2)
    got = C.copy()
    oracle.two_hop(oracle.Graph(xadj, adj, vw=vw, ew=ew), got, Wc.copy(), U, 5, 2)
    assert list(got) == list(want)


# Round tags spelled out from their ASCII names ("LPClustr", "LPRefine",
# "TieBrekr"), independently of the oracle's own constants.
TAG_CLUSTER = int.from_bytes(b"LPClustr", "big")
TAG_REFINE = int.from_bytes(b"LPRefine", "big")
TAG_TIE = int.from_bytes(b"TieBrekr", "big")


def _rounds_restated(xadj, adj, ew, vw, label, lw, nlabels, cap, seed, tag, level, rounds, S):
    """LP rounds from their definition: round r uses key (seed, tag, level, r)
    and runs sub-rounds 0..S-1, each by enumeration."""
    for r in range(rounds):
        rk = bf.round_key(seed, tag, level, r)
        for s in range(S):
            label, lw = bf.subround(xadj, adj, ew, vw, label, lw, nlabels, cap, rk, S, s, TAG_TIE)
    return label, lw


def _level_case(seed):
    rng, xadj, adj, ew, vw = _tiny(700 + seed, n=int(np.random.default_rng(seed).integers(8, 14)),
                                   p=0.4, max_w=4)
    p = oracle.Params(seed=int(rng.integers(1, 2**40)), cluster_rounds=int(rng.integers(1, 6)),
                      refine_rounds=int(rng.integers(1, 6)), sub_rounds=int(rng.integers(1, 5)))
    return rng, xadj, adj, ew, vw, p, int(rng.integers(0, 6))


def _cluster_case(seed):
    rng, xadj, adj, ew, vw, p, level = _level_case(seed)
    return xadj, adj, ew, vw, p, level, int(rng.integers(int(vw.max()), 14))


def _refine_case(seed):
    rng, xadj, adj, ew, vw, p, level = _level_case(seed)
    n = len(xadj) - 1
    k = int(rng.integers(2, 5))
    part = rng.integers(0, k, n).astype(np.int32)
    B = np.bincount(part, weights=vw, minlength=k).astype(np.int64)
    l_max = int(B.max()) + int(rng.integers(0, 5))  # some blocks can take moves, some not
    return xadj, adj, ew, vw, p, level, k, part, B, l_max


def _cluster_restated(xadj, adj, ew, vw, p, level, U):
    n = len(xadj) - 1
    label, lw = _rounds_restated(xadj, adj, ew, vw, np.arange(n, dtype=np.int32), vw.copy(), n,
                                 np.full(n, U, np.int64), p.seed, TAG_CLUSTER, level,
                                 p.cluster_rounds, p.sub_rounds)
    if p.two_hop:
        label = _two_hop_restated(xadj, adj, ew, vw, label, lw, U, p.seed, level)
    return label


def _refine_restated(xadj, adj, ew, vw, p, level, k, part, B, l_max):
    return _rounds_restated(xadj, adj, ew, vw, part.copy(), B.copy(), k,
                            np.full(k, l_max, np.int64), p.seed, TAG_REFINE, level,
                            p.refine_rounds, p.sub_rounds)


@pytest.mark.parametrize("seed", range(10))
def test_cluster_level_by_restatement(seed):
    # one coarsening level's clustering: the LP rounds with the cluster keys,
    # then two-hop packing of what stayed alone
    xadj, adj, ew, vw, p, level, U = _cluster_case(seed)
    g = oracle.Graph(xadj, adj, vw=vw, ew=ew)
    for two_hop in (0, 1):
        p.two_hop = two_hop
        want = _cluster_restated(xadj, adj, ew, vw, p, level, U)
        assert list(oracle.cluster(g, U, p, level)) == list(want), two_hop


@pytest.mark.parametrize("seed", range(10))
def test_refine_level_by_restatement(seed):
    # k-way refinement: the same LP with blocks as labels, block weights as
    # label weights, L_max as every block's cap and the refinement keys
    xadj, adj, ew, vw, p, level, k, part, B, l_max = _refine_case(seed)
    want, want_B = _refine_restated(xadj, adj, ew, vw, p, level, k, part, B, l_max)
    got, got_B = part.copy(), B.copy()
    oracle.refine(oracle.Graph(xadj, adj, vw=vw, ew=ew), got, got_B, k, l_max, p, level)
    assert list(got) == list(want) and list(got_B) == list(want_B)


def test_level_restatements_exercise_moves():
    # the cases above are not vacuous: most of them move vertices
    moved_c = moved_r = 0
    for seed in range(10):
        xadj, adj, ew, vw, p, level, U = _cluster_case(seed)
        p.two_hop = 0
        lab = _cluster_restated(xadj, adj, ew, vw, p, level, U)
        moved_c += int(np.any(lab != np.arange(len(xadj) - 1)))
        case = _refine_case(seed)
        lab, _ = _refine_restated(*case)
        moved_r += int(np.any(lab != case[7]))
    assert moved_c >= 8 and moved_r >= 5, (moved_c, moved_r)


def _tie_vec(hv, xs):
    # the tie hash of many labels at once (uint64 arithmetic wraps)
    z = np.uint64(hv) ^ (xs + np.uint64(bf.GAMMA))
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return z >> np.uint64(32)


def test_label_breaks_ties_of_rating_and_tie_hash():
    # the third level of the rating order only decides when two labels have
    # the same rating and the same 32-bit tie hash: find such a pair and put
    # both next to u with equal weight
    hv = 0x1234_5678_9ABC_DEF0
    xs = np.arange(1 << 18, dtype=np.uint64)
    t = _tie_vec(hv, xs)
    order = np.argsort(t, kind="stable")
    dup = np.nonzero(t[order][1:] == t[order][:-1])[0]
    assert len(dup) > 0
    x1, x2 = sorted((int(order[dup[0]]), int(order[dup[0] + 1])))
    assert bf.tie(hv, x1) == bf.tie(hv, x2)
    xadj = np.array([0, 2, 3, 4], np.int64)
    adj = np.array([1, 2, 0, 0], np.int32)
    for first, second in ((x2, x1), (x1, x2)):  # either neighbour order
        label = np.array([0, first, second], np.int32)
        lw = np.zeros(x2 + 1, np.int64)
        lw[0] = lw[x1] = lw[x2] = 1
        g = oracle.Graph(xadj, adj)
        for rate in (oracle.rate_vertex, oracle.rate_vertex_sorted):
            moved, target, gain = rate(g, 0, label, lw, 10, hv=hv)
            assert moved and target == x1 and gain == 1, rate
