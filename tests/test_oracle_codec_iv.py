"""Pins for the oracle's interval + weight variant of the compressed format
(Section "Compression Scheme": interval encoding, compressed edge weights):
hand-derived bytes, equality with the pinned plain format when both features
are off, the byte count by an independent formula, exact round trips and
rejection of corrupt streams."""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _golden():
    rows = {}
    with open(os.path.join(GOLD, "compress_iv.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                p = line.split()
                rows[p[0]] = p[1:]
    n = int(rows["n"][0])
    nb = [dict() for _ in range(n)]
    for e in rows["edges"]:
        uv, w = e.split(":")
        u, v = map(int, uv.split("-"))
        nb[u][v] = nb[v][u] = int(w)
    return rows, _csr_from(nb)


def _csr_from(nb):
    n = len(nb)
    xadj = np.zeros(n + 1, np.int64)
    adj, ew = [], []
    for u in range(n):
        for v in sorted(nb[u]):
            adj.append(v)
            ew.append(nb[u][v])
        xadj[u + 1] = len(adj)
    return xadj, np.array(adj, np.int32), np.array(ew, np.int64)


def _hex(row):
    return bytes(int(h, 16) for h in row)


def test_golden_bytes():
    rows, (xadj, adj, ew) = _golden()
    n = len(xadj) - 1
    data, off = oracle.encode_ex(xadj, adj, ew, intervals=True)
    assert bytes(data) == _hex(rows["iv_w_bytes"])
    assert list(off) == [int(x) for x in rows["iv_w_off"]]
    x2, a2, w2 = oracle.decode_ex(n, data, off, len(adj), intervals=True, weighted=True)
    assert np.array_equal(x2, xadj) and np.array_equal(a2, adj) and np.array_equal(w2, ew)
    data, off = oracle.encode_ex(xadj, adj, None, intervals=True)
    assert bytes(data) == _hex(rows["iv_bytes"])
    assert list(off) == [int(x) for x in rows["iv_off"]]
    x2, a2, w2 = oracle.decode_ex(n, data, off, len(adj), intervals=True, weighted=False)
    assert np.array_equal(a2, adj) and (w2 == 1).all()
    data, off = oracle.encode_ex(xadj, adj, ew, intervals=False)
    assert bytes(data[: off[1]]) == _hex(rows["w_vertex0"])


def _star_run(leaves=25000):
    # a hub adjacent to 1..leaves (one run cut by every chunk boundary) and
    # a path through the leaves
    nb = [dict() for _ in range(leaves + 1)]
    for v in range(1, leaves + 1):
        nb[0][v] = nb[v][0] = 1 + v % 7
    for v in range(1, leaves):
        nb[v][v + 1] = nb[v + 1][v] = 2
    return _csr_from(nb)


def _graphs():
    rng = np.random.default_rng(5)
    out = {}
    for name, (xadj, adj) in {"gnm": synth.gnm(3000, 20000, 2), "rgg": synth.rgg2d(8000, 16.0, 3),
                              "rmat": synth.rmat(12, 16, seed=4)}.items():
        ew = np.zeros(len(adj), np.int64)
        n = len(xadj) - 1
        for u in range(n):  # symmetric random weights
            for e in range(xadj[u], xadj[u + 1]):
                v = int(adj[e])
                if v > u:
                    w = int(rng.integers(1, 1000))
                    ew[e] = w
                    f = xadj[v] + int(np.searchsorted(adj[xadj[v]:xadj[v + 1]], u))
                    ew[f] = w
        out[name] = (xadj, adj, ew)
    out["star"] = _star_run()
    return out


GRAPHS = _graphs()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_plain_variant_equals_pinned_format(name):
    xadj, adj, _ = GRAPHS[name]
    want, woff = oracle.encode(xadj, adj)
    got, off = oracle.encode_ex(xadj, adj, None, intervals=False)
    assert np.array_equal(got, want) and np.array_equal(off, woff)


def _vlen(x):
    return max(1, (int(x).bit_length() + 6) // 7)


def _signed(x, ref):
    return 2 * (x - ref) if x >= ref else 2 * (ref - x) + 1


def _size_by_formula(xadj, adj, ew, intervals):
    """Byte count written out from the format: header per vertex, chunk table,
    per chunk the interval count, interval pairs, residual codes and one
    signed weight difference per edge; terminal header."""
    n = len(xadj) - 1
    total = _vlen(xadj[n])
    for u in range(n):
        b, d = int(xadj[u]), int(xadj[u + 1] - xadj[u])
        total += _vlen(b)
        if d == 0:
            continue
        nch = 1 if d <= 10000 else -(-d // 1000)
        csz = d if nch == 1 else 1000
        total += 4 * (nch - 1)
        for j in range(nch):
            ids = [int(x) for x in adj[b + j * csz: b + min(d, (j + 1) * csz)]]
            ws = None if ew is None else [int(x) for x in ew[b + j * csz: b + min(d, (j + 1) * csz)]]
            runs, resid = [], []
            if intervals:
                for _, grp in itertools.groupby(enumerate(ids), key=lambda t: t[1] - t[0]):
                    grp = [i for i, _ in grp]
                    (runs if len(grp) >= 3 else resid).append(grp)
                resid = [i for g in resid for i in g]
                total += _vlen(len(runs))
            else:
                resid = list(range(len(ids)))
            order = []
            prev_end = None
            for g in runs:
                x = ids[g[0]]
                total += _vlen(_signed(x, u) if prev_end is None else x - prev_end - 2)
                total += _vlen(len(g) - 3)
                prev_end = ids[g[-1]]
                order += g
            for k, i in enumerate(resid):
                total += _vlen(_signed(ids[i], u) if k == 0 else ids[i] - ids[resid[k - 1]])
            order += resid
            if ws is not None:
                prev = 0
                for i in order:
                    total += _vlen(_signed(ws[i], prev))
                    prev = ws[i]
    return total


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("intervals", [False, True])
@pytest.mark.parametrize("weighted", [False, True])
def test_size_formula_and_round_trip(name, intervals, weighted):
    xadj, adj, ew = GRAPHS[name]
    w = ew if weighted else None
    data, off = oracle.encode_ex(xadj, adj, w, intervals=intervals)
    if name != "star":  # the formula's Python loops are slow on the 25 000-leaf star
        assert len(data) == _size_by_formula(xadj, adj, w, intervals)
    x2, a2, w2 = oracle.decode_ex(len(xadj) - 1, data, off, len(adj), intervals=intervals,
                                  weighted=weighted)
    assert np.array_equal(x2, xadj) and np.array_equal(a2, adj)
    assert np.array_equal(w2, ew) if weighted else (w2 == 1).all()


def test_size_formula_on_the_chunked_star():
    # the formula on the star's hub alone (intervals cut at every chunk)
    xadj, adj, ew = GRAPHS["star"]
    hub = (np.array([0, xadj[1]], np.int64), adj[: xadj[1]], ew[: xadj[1]])
    for intervals in (False, True):
        for w in (None, hub[2]):
            data, _ = oracle.encode_ex(hub[0], hub[1], w, intervals=intervals)
            assert len(data) == _size_by_formula(hub[0], hub[1], w, intervals)
    data, _ = oracle.encode_ex(hub[0], hub[1], None, intervals=True)
    # by hand: header 1 byte, chunk table 24 * 4; 25 chunks, each one
    # interval: count 1 byte, length code 997 in 2 bytes, start code
    # 2 (1 + 1000 j) in 1 byte (j = 0), 2 bytes (j = 1..8), 3 bytes
    # (j = 9..24); terminal header 25 000 in 3 bytes
    assert len(data) == 1 + 96 + 25 * (1 + 2) + (1 + 8 * 2 + 16 * 3) + 3


def test_intervals_pay_on_locality():
    # runs of consecutive ids: fewer bytes; without runs: at most one byte
    # (the interval count) more per chunk
    xadj, adj, _ = GRAPHS["star"]
    hub = (np.array([0, xadj[1]], np.int64), adj[: xadj[1]])
    for name, (xadj, adj) in (("rgg", GRAPHS["rgg"][:2]), ("hub", hub)):
        plain = len(oracle.encode_ex(xadj, adj, None, intervals=False)[0])
        iv = len(oracle.encode_ex(xadj, adj, None, intervals=True)[0])
        assert iv < plain, name
    xadj, adj, _ = GRAPHS["gnm"]
    nonempty = int(np.sum(np.diff(xadj) > 0))
    plain = len(oracle.encode_ex(xadj, adj, None, intervals=False)[0])
    iv = len(oracle.encode_ex(xadj, adj, None, intervals=True)[0])
    assert plain <= iv <= plain + nonempty


def test_rejects_corrupt_streams():
    rows, (xadj, adj, ew) = _golden()
    n = len(xadj) - 1
    data, off = oracle.encode_ex(xadj, adj, ew, intervals=True)

    def bad(mutate):
        d = data.copy()
        mutate(d)
        with pytest.raises(ValueError):
            oracle.decode_ex(n, d, off, len(adj), intervals=True, weighted=True)

    bad(lambda d: d.__setitem__(3, 0x20))   # u=0's interval longer than its six ids
    bad(lambda d: d.__setitem__(1, 0x03))   # three intervals announced in six ids
    bad(lambda d: d.__setitem__(8, 0x04))   # residual 2 lies inside the interval
    bad(lambda d: d.__setitem__(10, 0x00))  # residual gap 0: duplicate id
    bad(lambda d: d.__setitem__(5, 0x0b))   # weight 5 - 5 = 0: not positive
    bad(lambda d: d.__setitem__(11, 0x82))  # truncated weight VarInt
    # the plain weighted variant: a weight that drops below one
    d, o = oracle.encode_ex(xadj, adj, ew, intervals=False)
    d = d.copy()
    d[4] = 0x0b  # vertex 0, second weight 5 - 5
    with pytest.raises(ValueError):
        oracle.decode_ex(n, d, o, len(adj), intervals=False, weighted=True)


def test_coarse_levels_round_trip_with_weights():
    # coarse levels carry node and edge weights; their adjacency and edge
    # weights round-trip through the weighted format (coarse-level
    # compression, the row after interval encoding)
    xadj, adj = synth.rgg2d(20000, 16.0, 7)
    g = oracle.Graph(xadj, adj)
    for level in range(3):
        C = oracle.cluster(g, 40 * (level + 1), oracle.Params(seed=2), level)
        g, _ = oracle.contract(g, C)
        for intervals in (False, True):
            data, off = oracle.encode_ex(g.xadj, g.adj, g.ew, intervals=intervals)
            x2, a2, w2 = oracle.decode_ex(g.n, data, off, len(g.adj), intervals=intervals,
                                          weighted=True)
            assert np.array_equal(x2, g.xadj) and np.array_equal(a2, g.adj)
            assert np.array_equal(w2, g.ew)
            assert len(data) == _size_by_formula(g.xadj, g.adj, g.ew, intervals)


def test_rejects_chunks_that_run_backwards():
    # star with 10 001 leaves, intervals on: every chunk is one interval.
    # Chunk 0 takes 4 bytes after the 1-byte header and the 40-byte table
    # (count 01, start 2*1 = 02, length 997 - 3 in two bytes), so chunk 1
    # starts at byte 45 with count 01 and start VarInt(2 * 1001) in two
    # bytes; VarInt(2 * 500) also takes two bytes and sends chunk 1 back over
    # ids chunk 0 already holds
    leaves = 10001
    nb = [dict() for _ in range(leaves + 1)]
    for v in range(1, leaves + 1):
        nb[0][v] = nb[v][0] = 1
    xadj, adj, _ = _csr_from(nb)
    data, off = oracle.encode_ex(xadj, adj, None, intervals=True)
    assert data[45] == 1 and bytes(data[46:48]) == oracle.varint(2 * 1001)
    oracle.decode_ex(leaves + 1, data, off, len(adj), intervals=True)
    bad = data.copy()
    bad[46:48] = np.frombuffer(oracle.varint(2 * 500), np.uint8)
    with pytest.raises(ValueError):
        oracle.decode_ex(leaves + 1, bad, off, len(adj), intervals=True)
