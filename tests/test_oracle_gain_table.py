"""Pins for the oracle's space-efficient gain table (Section "Space-Efficient
Gain Tables"): every affinity equals a brute-force recount after building and
after each move of a random sequence, sparse tables hold exactly the blocks
with non-zero affinity and keep every key on its probe path, and the memory
footprint and value widths follow the stated layout."""
import numpy as np
import pytest

import oracle
from tests import _brute as bf


def _affinity(xadj, adj, ew, part, v, b):
    return sum(int(ew[e]) for e in range(xadj[v], xadj[v + 1]) if part[adj[e]] == b)


def _case(seed):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(10, 40))
    xadj, adj, ew, vw = bf.random_graph(rng, n, float(rng.uniform(0.1, 0.5)), max_w=300)
    k = int(rng.integers(2, 9))
    part = rng.integers(0, k, n).astype(np.int32)
    return rng, xadj, adj, ew, vw, k, part


def _check_all(t, xadj, adj, ew, part, k):
    n = len(xadj) - 1
    for v in range(n):
        for b in range(k):
            assert t.get(v, b) == _affinity(xadj, adj, ew, part, v, b), (v, b)
        lay = t.layout(v)
        if not lay["dense"] and lay["cap"]:
            nonzero = sum(_affinity(xadj, adj, ew, part, v, b) > 0 for b in range(k))
            assert lay["stored"] == nonzero, v
    assert t.check() == 0


@pytest.mark.parametrize("seed", range(12))
def test_affinities_after_random_moves(seed):
    rng, xadj, adj, ew, vw, k, part = _case(seed)
    g = oracle.Graph(xadj, adj, vw=vw, ew=ew)
    t = oracle.GainTable(g, part, k)
    _check_all(t, xadj, adj, ew, part, k)
    n = len(xadj) - 1
    for step in range(120):
        u = int(rng.integers(0, n))
        to = int(rng.integers(0, k))
        t.move(u, int(part[u]), to)
        part[u] = to
        if step % 10 == 9:
            _check_all(t, xadj, adj, ew, part, k)
    _check_all(t, xadj, adj, ew, part, k)


def test_cases_mix_dense_and_sparse_vertices():
    dense = sparse = 0
    for seed in range(12):
        _, xadj, adj, ew, vw, k, part = _case(seed)
        t = oracle.GainTable(oracle.Graph(xadj, adj, vw=vw, ew=ew), part, k)
        for v in range(len(xadj) - 1):
            lay = t.layout(v)
            dense += lay["dense"]
            sparse += not lay["dense"] and lay["cap"] > 0
    assert dense >= 50 and sparse >= 50, (dense, sparse)


def _width(total):
    for w in (1, 2, 4, 8):
        if total < 1 << (8 * w):
            return w
    raise AssertionError


@pytest.mark.parametrize("seed", range(6))
def test_footprint_and_widths(seed):
    _, xadj, adj, ew, vw, k, part = _case(seed)
    g = oracle.Graph(xadj, adj, vw=vw, ew=ew)
    t = oracle.GainTable(g, part, k)
    want = 0
    for v in range(len(xadj) - 1):
        d = int(xadj[v + 1] - xadj[v])
        total = int(ew[xadj[v]:xadj[v + 1]].sum())
        w = _width(total)
        lay = t.layout(v)
        assert lay["width"] == w and lay["dense"] == (d > k)
        if d > k:
            cap = k
            want += k * w
        elif d > 0:
            cap = 1 << (2 * d - 1).bit_length()  # smallest power of two >= 2 d
            want += cap * (4 + w)
        else:
            cap = 0
        assert lay["cap"] == cap, v
    assert t.bytes() == want
    # O(m): at most 2 (4 + 8) bytes per adjacency entry plus 8 bytes per block
    # of each dense vertex
    assert t.bytes() <= 24 * len(adj) + 8 * k * (len(xadj) - 1)


def test_widths_grow_with_incident_weight():
    # a star whose leaves carry one edge each: the hub's total weight picks
    # its width, and a single deletion empties a leaf's table
    for w_edge, hub_width in ((1, 1), (200, 2), (70000, 4), (1 << 33, 8)):
        leaves = 4
        xadj = np.array([0, leaves] + [leaves + i + 1 for i in range(leaves)], np.int64)
        adj = np.array([1, 2, 3, 4] + [0] * leaves, np.int32)
        ew = np.full(2 * leaves, w_edge, np.int64)
        part = np.array([0, 1, 1, 2, 2], np.int32)
        g = oracle.Graph(xadj, adj, ew=ew)
        t = oracle.GainTable(g, part, 3)
        assert t.layout(0)["width"] == hub_width
        assert t.get(0, 1) == 2 * w_edge and t.get(0, 2) == 2 * w_edge and t.get(0, 0) == 0
        t.move(0, 0, 1)  # every leaf's only affinity moves from block 0 to 1
        assert all(t.get(v, 0) == 0 and t.get(v, 1) == w_edge for v in range(1, 5))
        assert all(t.layout(v)["stored"] == 1 for v in range(1, 5)) and t.check() == 0
