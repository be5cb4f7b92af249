"""Pins for the oracle's compressed adjacency format (Section "Compression
Scheme"): hand-derived bytes, the chunk layout, exact round trips, the byte
count by formula and rejection of corrupt streams."""
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lines(name):
    with open(os.path.join(GOLD, name)) as f:
        return [l.split() for l in f if l.strip() and not l.startswith("#")]


def test_varint_golden():
    for row in _lines("varint.txt"):
        value, want = int(row[0]), bytes(int(h, 16) for h in row[1:])
        assert oracle.varint(value) == want, value


def _csr(n, edges):
    nb = [[] for _ in range(n)]
    for u, v in edges:
        nb[u].append(v)
        nb[v].append(u)
    xadj = np.zeros(n + 1, np.int64)
    adj = []
    for u in range(n):
        adj += sorted(nb[u])
        xadj[u + 1] = len(adj)
    return xadj, np.array(adj, np.int32)


def test_compress_5v_golden():
    rows = {r[0]: r[1:] for r in _lines("compress_5v.txt")}
    n = int(rows["n"][0])
    edges = [tuple(map(int, e.split("-"))) for e in rows["edges"]]
    xadj, adj = _csr(n, edges)
    data, off = oracle.encode(xadj, adj)
    assert bytes(data) == bytes(int(h, 16) for h in rows["bytes"])
    assert list(off) == [int(x) for x in rows["off"]]
    x2, a2 = oracle.decode(n, data, off, len(adj))
    assert np.array_equal(x2, xadj) and np.array_equal(a2, adj)


def test_compress_star_chunks_golden():
    rows = {r[0]: r[1:] for r in _lines("compress_star.txt")}
    leaves = int(rows["leaves"][0])
    xadj, adj = _csr(leaves + 1, [(0, v) for v in range(1, leaves + 1)])
    data, off = oracle.encode(xadj, adj)
    assert int(off[1] - off[0]) == int(rows["vertex0_bytes"][0])
    table = np.frombuffer(bytes(data[1:41]), dtype="<u4")
    assert list(table) == [int(x) for x in rows["table"]]
    assert data[0] == 0 and data[41] == 2 and all(data[42:1041] == 1)
    # leaf 1: header = first edge id 10001, first neighbour 0 < 1 -> 2*1+1
    p = int(off[1])
    assert bytes(data[p:p + 3]) == oracle.varint(10001) + oracle.varint(3)
    x2, a2 = oracle.decode(leaves + 1, data, off, len(adj))
    assert np.array_equal(x2, xadj) and np.array_equal(a2, adj)


def _size_by_formula(xadj, adj):
    def vlen(x):
        return max(1, (int(x).bit_length() + 6) // 7)

    total = vlen(xadj[-1])
    for u in range(len(xadj) - 1):
        nb = [int(v) for v in adj[xadj[u]:xadj[u + 1]]]
        total += vlen(xadj[u])
        d = len(nb)
        if d == 0:
            continue
        csz = 1000 if d > 10000 else d
        total += 4 * (-(-d // csz) - 1)
        for i, v in enumerate(nb):
            if i % csz == 0:
                total += vlen(2 * abs(v - u) + (v < u))
            else:
                total += vlen(v - nb[i - 1])
    return total


@pytest.mark.parametrize("kind", ["gnm", "rgg", "rmat"])
def test_roundtrip_and_size(kind):
    if kind == "gnm":
        xadj, adj = synth.gnm(3000, 20000, 7)
    elif kind == "rgg":
        xadj, adj = synth.rgg2d(5000, 16.0, 3)
    else:
        xadj, adj = synth.rmat(14, 16, seed=5)
    data, off = oracle.encode(xadj, adj)
    assert len(data) == _size_by_formula(xadj, adj)
    x2, a2 = oracle.decode(len(xadj) - 1, data, off, len(adj))
    assert np.array_equal(x2, xadj) and np.array_equal(a2, adj)


def test_roundtrip_high_degree_mixed():
    # a hub adjacent to every other vertex plus a path: chunked + plain lists
    n = 25001
    edges = [(0, v) for v in range(1, n)] + [(v, v + 1) for v in range(1, n - 1)]
    xadj, adj = _csr(n, edges)
    data, off = oracle.encode(xadj, adj)
    assert len(data) == _size_by_formula(xadj, adj)
    x2, a2 = oracle.decode(n, data, off, len(adj))
    assert np.array_equal(x2, xadj) and np.array_equal(a2, adj)


def test_decode_rejects_corruption():
    xadj, adj = synth.gnm(200, 1000, 2)
    data, off = oracle.encode(xadj, adj)
    n = len(xadj) - 1
    # truncated VarInt: set the continuation bit on the last byte of vertex 0
    bad = data.copy()
    bad[int(off[1]) - 1] |= 0x80
    with pytest.raises(ValueError):
        oracle.decode(n, bad, off, len(adj))
    # neighbour id out of range: a huge first-neighbour offset
    u = 5
    p = int(off[u]) + len(oracle.varint(int(xadj[u])))
    bad2 = np.concatenate([data[:p], np.frombuffer(oracle.varint(2 * 10**6), np.uint8),
                           data[p + 1:]]).astype(np.uint8)
    off2 = off.copy()
    off2[u + 1:] += len(oracle.varint(2 * 10**6)) - 1
    with pytest.raises(ValueError):
        oracle.decode(n, bad2, off2, len(adj))


def test_decode_rejects_bad_first_header_and_unordered_chunks():
    xadj, adj = synth.gnm(200, 1000, 2)
    data, off = oracle.encode(xadj, adj)
    bad = data.copy()
    bad[0] = 0x01  # the first neighbourhood must start at edge id 0
    with pytest.raises(ValueError):
        oracle.decode(len(xadj) - 1, bad, off, len(adj))
    # every header one higher (edge ids counted from 1): the records still
    # agree with each other, only the first header shows the shift
    shifted, soff = oracle.encode(xadj + 1, np.concatenate([[0], adj]).astype(np.int32))
    with pytest.raises(ValueError):
        oracle.decode(len(xadj) - 1, shifted, soff, len(adj) + 1)
    # star with 10 001 leaves: chunk 1 starts at byte 1041 with VarInt(2 * 1001)
    # (two bytes); VarInt(2 * 500) also takes two bytes and sends chunk 1 back
    # below the end of chunk 0
    leaves = 10001
    xadj, adj = _csr(leaves + 1, [(0, v) for v in range(1, leaves + 1)])
    data, off = oracle.encode(xadj, adj)
    assert bytes(data[1041:1043]) == oracle.varint(2 * 1001)
    bad = data.copy()
    bad[1041:1043] = np.frombuffer(oracle.varint(2 * 500), np.uint8)
    with pytest.raises(ValueError):
        oracle.decode(leaves + 1, bad, off, len(adj))
