"""GPU path against the oracle, element by element, through the C-ABI.

Every comparison is exact: the method is integer-only (int64 sums on coarse
levels) and deterministic, so clusterings, coarse graphs, partitions, cuts
and imbalances must be bit-identical to the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402


def _star_path(leaves=25000):
    # a hub adjacent to every leaf plus a path through the leaves: the hub is
    # chunked in the compressed format and rated by the huge tier
    n = leaves + 1
    nb = [[] for _ in range(n)]
    for v in range(1, n):
        nb[0].append(v)
        nb[v].append(0)
    for v in range(1, n - 1):
        nb[v].append(v + 1)
        nb[v + 1].append(v)
    xadj = np.zeros(n + 1, np.int64)
    adj = []
    for u in range(n):
        adj += sorted(nb[u])
        xadj[u + 1] = len(adj)
    return xadj, np.array(adj, np.int32)


def _multi_star(hubs=4, leaves=10500):
    # several hubs above the chunking threshold (huge tier, each in its own
    # sub-round most of the time), their leaves on one path, hubs in a clique
    n = hubs * (leaves + 1)
    nb = [set() for _ in range(n)]

    def link(a, b):
        nb[a].add(b)
        nb[b].add(a)

    for h in range(hubs):
        base = h * (leaves + 1)
        for v in range(base + 1, base + leaves + 1):
            link(base, v)
        for h2 in range(h + 1, hubs):
            link(base, h2 * (leaves + 1))
    leaves_all = [v for v in range(n) if v % (leaves + 1) != 0]
    for a, b in zip(leaves_all[:-1], leaves_all[1:]):
        link(a, b)
    xadj = np.zeros(n + 1, np.int64)
    adj = []
    for u in range(n):
        adj += sorted(nb[u])
        xadj[u + 1] = len(adj)
    return xadj, np.array(adj, np.int32)


GRAPHS = {
    "gnm": lambda: synth.gnm(3000, 24000, 3),
    "rgg": lambda: synth.rgg2d(5000, 16.0, 2),
    "rmat": lambda: synth.rmat(13, 16, seed=4),
    "star": _star_path,
}


@pytest.fixture(scope="module", params=list(GRAPHS))
def graph(request):
    xadj, adj = GRAPHS[request.param]()
    return request.param, xadj, adj


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _host(t):
    return t.cpu().numpy()


def test_compress_bytes_equal_oracle(graph):
    name, xadj, adj = graph
    g = tp.graph_from_csr(xadj, adj)
    z = g.compress()
    data, off = z.export_compressed()
    want_data, want_off = oracle.encode(xadj, adj)
    assert np.array_equal(_host(off).astype(np.uint64), want_off)
    assert np.array_equal(_host(data), want_data)
    x2, a2, _, _ = z.decompress().export_csr()
    assert np.array_equal(_host(x2), xadj) and np.array_equal(_host(a2), adj)


def test_from_compressed_validates():
    xadj, adj = synth.gnm(500, 3000, 9)
    data, off = oracle.encode(xadj, adj)
    z = tp.graph_from_compressed(len(xadj) - 1, data, off)
    x2, a2, _, _ = z.decompress().export_csr()
    assert np.array_equal(_host(x2), xadj) and np.array_equal(_host(a2), adj)
    bad = data.copy()
    bad[int(off[1]) - 1] |= 0x80  # truncate the last VarInt of vertex 0
    with pytest.raises(tp.TpError) as e:
        tp.graph_from_compressed(len(xadj) - 1, bad, off)
    assert e.value.code == 4
    bad = data.copy()
    p = int(off[7]) + len(oracle.varint(int(xadj[7])))
    bad[p + 1] = 0  # a zero gap: duplicate neighbour
    with pytest.raises(tp.TpError) as e:
        tp.graph_from_compressed(len(xadj) - 1, bad, off)
    assert e.value.code == 4


def test_wide_offsets(monkeypatch):
    """u64 offsets (chosen from 4 GiB of stream on; forced here on small
    graphs) give the same stream, clusterings and partitions as u32 ones."""
    monkeypatch.setenv("TP_OFFSETS_U64", "1")
    for xadj, adj in (_star_path(12000), synth.rmat(12, 16, seed=5)):
        n = len(xadj) - 1
        og = oracle.Graph(xadj, adj)
        want_data, want_off = oracle.encode(xadj, adj)
        want_c = oracle.cluster(og, 30, oracle.Params(seed=5), 0)
        want_p, _ = oracle.partition(og, 8, 0.03, oracle.Params(seed=5))
        for z in (tp.graph_from_csr(xadj, adj).compress(),
                  tp.graph_from_compressed(n, want_data, want_off)):
            inf = z.info()
            assert inf["compressed"] and inf["bytes"] == inf["stream_bytes"] + 8 * (n + 1)
            data, off = z.export_compressed()
            assert np.array_equal(_host(off).astype(np.uint64), want_off)
            assert np.array_equal(_host(data), want_data)
            x2, a2, _, _ = z.decompress().export_csr()
            assert np.array_equal(_host(x2), xadj) and np.array_equal(_host(a2), adj)
            got = tp.lp_cluster(z, 30, tp.default_params(seed=5), 0)
            assert np.array_equal(_host(got), want_c)
            part, _ = tp.partition(z, 8, 0.03, tp.default_params(seed=5))
            assert np.array_equal(_host(part), want_p)
            z.check()


def test_rejects_invalid_csr():
    xadj, adj = synth.gnm(100, 400, 1)
    bad = adj.copy()
    bad[0], bad[1] = bad[1], bad[0]  # unsorted neighbourhood
    with pytest.raises(tp.TpError) as e:
        tp.graph_from_csr(xadj, bad)
    assert e.value.code == 1


@pytest.mark.parametrize("compressed", [False, True])
def test_lp_subround_parity(graph, compressed):
    name, xadj, adj = graph
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
    og = oracle.Graph(xadj, adj)
    n = len(xadj) - 1
    U = 40
    label = np.arange(n, dtype=np.int32)
    lw = np.ones(n, np.int64)
    dl, dw = _dev(label), _dev(lw)
    S = 8
    for r in range(2):
        rk = oracle.round_key(7, oracle.tag(oracle.TAG_CLUSTER), 0, r)
        for s in range(S):
            oracle.lp_subround(og, label, lw, n, U, None, rk, S, s)
            tp.lp_subround(g, dl, dw, U, rk, S, s)
            assert np.array_equal(_host(dl), label), (name, r, s)
            assert np.array_equal(_host(dw), lw), (name, r, s)
    g.check()


def test_lp_subround_contested_targets():
    # every leaf of a star wants the hub's label; the cap admits only a few,
    # so approval must pick the longest (gain desc, id asc) prefix
    xadj, adj = _star_path(3000)
    n = len(xadj) - 1
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    label = np.zeros(n, np.int32)
    label[1:] = np.arange(1, n)
    lw = np.zeros(n, np.int64)
    np.add.at(lw, label, 1)
    for cap in (5, 37, 200):
        lab, w = label.copy(), lw.copy()
        dl, dw = _dev(lab), _dev(w)
        rk = oracle.round_key(3, 11, 0, cap)
        oracle.lp_subround(og, lab, w, n, cap, None, rk, 2, 1)
        tp.lp_subround(g, dl, dw, cap, rk, 2, 1)
        assert np.array_equal(_host(dl), lab) and np.array_equal(_host(dw), w)


@pytest.mark.parametrize("compressed", [False, True])
def test_cluster_parity(graph, compressed):
    name, xadj, adj = graph
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
    og = oracle.Graph(xadj, adj)
    for U, level in ((30, 0), (7, 3)):
        want = oracle.cluster(og, U, oracle.Params(seed=5), level)
        got = tp.lp_cluster(g, U, tp.default_params(seed=5), level)
        assert np.array_equal(_host(got), want), (name, U)
    g.check()


def test_contract_parity(graph):
    name, xadj, adj = graph
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    C = oracle.cluster(og, 25, oracle.Params(), 0)
    want_g, want_map = oracle.contract(og, C)
    for gg in (g, g.compress()):
        cg, mp = tp.contract(gg, _dev(C))
        x, a, vw, ew = (_host(t) for t in cg.export_csr())
        assert np.array_equal(_host(mp), want_map)
        assert np.array_equal(x, want_g.xadj) and np.array_equal(a, want_g.adj)
        assert np.array_equal(vw, want_g.vw) and np.array_equal(ew, want_g.ew)
    # second level: weighted contraction of the coarse graph
    C2 = oracle.cluster(want_g, 60, oracle.Params(), 1)
    want2, map2 = oracle.contract(want_g, C2)
    cg = tp.graph_from_csr(want_g.xadj, want_g.adj, want_g.vw, want_g.ew)
    cg2, mp2 = tp.contract(cg, _dev(C2))
    x, a, vw, ew = (_host(t) for t in cg2.export_csr())
    assert np.array_equal(_host(mp2), map2)
    assert np.array_equal(x, want2.xadj) and np.array_equal(a, want2.adj)
    assert np.array_equal(vw, want2.vw) and np.array_equal(ew, want2.ew)


def _coarse(xadj, adj, U=20, levels=2):
    g = oracle.Graph(xadj, adj)
    for lv in range(levels):
        C = oracle.cluster(g, U * (lv + 1), oracle.Params(), lv)
        g, _ = oracle.contract(g, C)
    return g


@pytest.mark.parametrize("k", [2, 3, 8, 13])
def test_initial_partition_parity(graph, k):
    name, xadj, adj = graph
    og = _coarse(xadj, adj)
    l_max = oracle.block_cap(int(og.vw.sum()), k, 30000)
    want = oracle.initial_partition(og, k, l_max, oracle.Params(seed=2))
    g = tp.graph_from_csr(og.xadj, og.adj, og.vw, og.ew)
    got = tp.initial_partition(g, k, l_max, tp.default_params(seed=2))
    assert np.array_equal(_host(got), want), (name, k)


@pytest.mark.parametrize("compressed", [False, True])
def test_refine_and_rebalance_parity(graph, compressed):
    name, xadj, adj = graph
    og = oracle.Graph(xadj, adj)
    n = len(xadj) - 1
    k = 6
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
    # a deliberately unbalanced start: block 0 is twice its share
    part = (np.arange(n) * k // n).astype(np.int32)
    part[: n // 6] = 0
    part[n // 6: n // 3] = 0
    l_max = oracle.block_cap(n, k, 30000)
    B = oracle.block_weights(og, part, k)
    want = part.copy()
    oracle.rebalance(og, want, B, k, l_max)
    got = _dev(part)
    assert tp.rebalance(g, k, l_max, got) == bool(B.max() <= l_max)
    assert np.array_equal(_host(got), want)
    oracle.refine(og, want, B, k, l_max, oracle.Params(seed=4), 2)
    tp.lp_refine(g, k, l_max, got, tp.default_params(seed=4), level=2)
    assert np.array_equal(_host(got), want)
    cut, Bg = tp.metrics(g, got, k)
    assert cut == oracle.cut(og, want) and np.array_equal(Bg, oracle.block_weights(og, want, k))


def _partition_both(xadj, adj, k, seed=1, compressed=False, params=None):
    og = oracle.Graph(xadj, adj)
    want, wst = oracle.partition(og, k, 0.03, oracle.Params(seed=seed))
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
    part, st = tp.partition(g, k, 0.03, params or tp.default_params(seed=seed))
    return want, wst, _host(part), st


@pytest.mark.parametrize("compressed", [False, True])
def test_partition_config1_parity(compressed):
    # plain method, small: G(n,m), n = 2^14, m = 2^17, k = 8, eps = 0.03, seed 1
    xadj, adj = synth.gnm(1 << 14, 1 << 17, 1)
    want, wst, got, st = _partition_both(xadj, adj, 8, 1, compressed)
    assert np.array_equal(got, want)
    for key in ("cut", "max_block_weight", "l_max", "u_max", "imbalance", "levels", "balanced",
                "level_n", "level_m2"):
        assert st[key] == wst[key], key


@pytest.mark.parametrize("kind,k", [("rgg", 16), ("rmat", 32), ("gnm", 3)])
@pytest.mark.parametrize("compressed", [False, True])
def test_partition_parity_families(kind, k, compressed):
    if kind == "rgg":
        xadj, adj = synth.rgg2d(1 << 16, 16.0, 3)
    elif kind == "rmat":
        xadj, adj = synth.rmat(15, 16, seed=2)
    else:
        xadj, adj = synth.gnm(5000, 20000, 8)
    want, wst, got, st = _partition_both(xadj, adj, k, 3, compressed)
    assert np.array_equal(got, want)
    assert st["cut"] == wst["cut"] and st["level_n"] == wst["level_n"]


def _degree_boundaries(leaves=30000, seed=12):
    # hubs whose degrees sit on both sides of every tier boundary and of the
    # chunking threshold (10 000 / 10 001 neighbours, chunks of 1 000), over
    # leaves joined by a path and random edges
    degs = [1, 31, 32, 33, 63, 64, 65, 255, 256, 257, 511, 512, 513, 1000, 1024, 1025, 2048,
            2049, 4096, 4097, 9999, 10000, 10001, 10999, 11000]
    h = len(degs)
    rng = np.random.default_rng(seed)
    edges = set()
    for i, d in enumerate(degs):
        for v in rng.choice(leaves, d, replace=False):
            edges.add((i, h + int(v)))
    for v in range(leaves - 1):
        edges.add((h + v, h + v + 1))
    for a, b in rng.integers(0, leaves, size=(2 * leaves, 2)):
        if a != b:
            edges.add((h + int(min(a, b)), h + int(max(a, b))))
    n = h + leaves
    nb = [[] for _ in range(n)]
    for a, b in edges:
        nb[a].append(b)
        nb[b].append(a)
    xadj = np.zeros(n + 1, np.int64)
    xadj[1:] = np.cumsum([len(x) for x in nb])
    adj = np.concatenate([np.sort(np.array(x, np.int32)) for x in nb]).astype(np.int32)
    assert list(np.diff(xadj)[:h]) == degs
    return xadj, adj


@pytest.mark.parametrize("compressed", [False, True])
def test_degree_boundaries(compressed):
    xadj, adj = _degree_boundaries()
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
        data, off = g.export_compressed()
        want_data, want_off = oracle.encode(xadj, adj)
        assert np.array_equal(_host(off).astype(np.uint64), want_off)
        assert np.array_equal(_host(data), want_data)
    for U, level in ((40, 0), (20000, 1)):
        want = oracle.cluster(og, U, oracle.Params(seed=11), level)
        got = tp.lp_cluster(g, U, tp.default_params(seed=11), level)
        assert np.array_equal(_host(got), want), U
    want, wst = oracle.partition(og, 16, 0.03, oracle.Params(seed=11))
    part, st = tp.partition(g, 16, 0.03, tp.default_params(seed=11))
    assert np.array_equal(_host(part), want) and st["cut"] == wst["cut"]
    g.check()


@pytest.mark.parametrize("compressed", [False, True])
def test_direct_rounds_with_several_hubs(compressed):
    """Several chunked hubs rated in sub-round buckets (their chunk and table
    segment items listed per round) against the oracle."""
    xadj, adj = _multi_star()
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
    for use_graphs in (0, 1):
        p = tp.default_params(seed=3, use_graphs=use_graphs)
        want = oracle.cluster(og, 40, oracle.Params(seed=3), 0)
        assert np.array_equal(_host(tp.lp_cluster(g, 40, p, 0)), want), use_graphs
        want, wst = oracle.partition(og, 6, 0.03, oracle.Params(seed=3))
        part, st = tp.partition(g, 6, 0.03, p)
        assert np.array_equal(_host(part), want) and st["cut"] == wst["cut"], use_graphs
    g.check()


@pytest.mark.parametrize("compressed", [False, True])
def test_direct_rounds_equal_oracle(graph, compressed):
    """Rounds launched kernel by kernel (as on levels above 2^19 vertices,
    with every tier's vertices bucketed by sub-round once per round) give the
    same clustering and partition as the oracle; use_graphs = 0 forces that
    path on these small graphs."""
    name, xadj, adj = graph
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
    p = tp.default_params(seed=5, use_graphs=0)
    want = oracle.cluster(og, 30, oracle.Params(seed=5), 0)
    assert np.array_equal(_host(tp.lp_cluster(g, 30, p, 0)), want), name
    want, wst = oracle.partition(og, 8, 0.03, oracle.Params(seed=5))
    part, st = tp.partition(g, 8, 0.03, p)
    assert np.array_equal(_host(part), want) and st["cut"] == wst["cut"], name
    g.check()


def test_performance_knobs_do_not_change_results():
    xadj, adj = synth.rmat(14, 16, seed=6)
    og = oracle.Graph(xadj, adj)
    want, _ = oracle.partition(og, 12, 0.03, oracle.Params(seed=9))
    g = tp.graph_from_csr(xadj, adj)
    z = g.compress()
    rng = np.random.default_rng(0)
    for trial in range(4):
        p = tp.default_params(seed=9, tier_lane=int(rng.choice([0, 8, 16, 32])),
                              tier_small=int(rng.choice([1, 16, 32, 64])),
                              tier_mid=int(rng.choice([64, 200, 1000])),
                              warps_per_block=int(rng.choice([2, 4, 8, 16])),
                              use_graphs=int(rng.choice([0, 1])))
        for gg in (g, z):
            part, _ = tp.partition(gg, 12, 0.03, p)
            assert np.array_equal(_host(part), want), trial


def _sym_weights(xadj, adj, rng, hi):
    ew = np.zeros(len(adj), np.int64)
    for u in range(len(xadj) - 1):
        for e in range(xadj[u], xadj[u + 1]):
            v = int(adj[e])
            if v > u:
                w = int(rng.integers(1, hi))
                ew[e] = w
                ew[xadj[v] + int(np.searchsorted(adj[xadj[v]:xadj[v + 1]], u))] = w
    return ew


def test_partition_parameter_extremes():
    # eps = 0 (cluster cap 1: no level coarsens), k = 1024 on 2 500 vertices,
    # k = n, and an input graph with node and edge weights
    xadj, adj = synth.gnm(2500, 9000, 6)
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    for k, eps in ((5, 0.0), (1024, 0.03), (2500, 0.03)):
        want, wst = oracle.partition(og, k, eps, oracle.Params(seed=8))
        part, st = tp.partition(g, k, eps, tp.default_params(seed=8))
        assert np.array_equal(_host(part), want), (k, eps)
        assert st["cut"] == wst["cut"] and st["level_n"] == wst["level_n"], (k, eps)
    rng = np.random.default_rng(4)
    xadj, adj = synth.rgg2d(3000, 12.0, 9)
    vw = rng.integers(1, 6, len(xadj) - 1).astype(np.int64)
    ew = _sym_weights(xadj, adj, rng, 10)
    want, wst = oracle.partition(oracle.Graph(xadj, adj, vw=vw, ew=ew), 7, 0.03,
                                 oracle.Params(seed=8))
    part, st = tp.partition(tp.graph_from_csr(xadj, adj, vw, ew), 7, 0.03,
                            tp.default_params(seed=8))
    assert np.array_equal(_host(part), want) and st["cut"] == wst["cut"]


def test_edge_cases():
    # empty graph, isolated vertices only, k = 1, k > n
    empty = tp.graph_from_csr(np.zeros(1, np.int64), np.zeros(0, np.int32))
    part, st = tp.partition(empty, 4)
    assert part.numel() == 0 and st["cut"] == 0
    iso_x = np.zeros(1001, np.int64)
    iso_a = np.zeros(0, np.int32)
    want, wst = oracle.partition(oracle.Graph(iso_x, iso_a), 4, 0.03, oracle.Params())
    part, st = tp.partition(tp.graph_from_csr(iso_x, iso_a), 4)
    assert np.array_equal(_host(part), want) and st["balanced"] == wst["balanced"]
    xadj, adj = synth.gnm(300, 1200, 4)
    part, st = tp.partition(tp.graph_from_csr(xadj, adj), 1)
    assert not _host(part).any() and st["cut"] == 0
    want, wst = oracle.partition(oracle.Graph(xadj, adj), 400, 0.03, oracle.Params())
    part, st = tp.partition(tp.graph_from_csr(xadj, adj), 400)
    assert np.array_equal(_host(part), want)
