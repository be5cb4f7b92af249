"""The interval + edge-weight stream on the GPU (tp_encode_ex,
tp_graph_from_stream_ex) against the oracle's encoder and decoder
(oracle/codec_iv.c): byte-identical streams and offsets with and without
intervals and weights, including a hub stored in chunks; the plain stream of
tp_graph_compress when both are off; exact round trips; corrupt streams
refused; a decoded weighted graph partitions like the oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402


def _sym_weights(xadj, adj, seed):
    rng = np.random.default_rng(seed)
    n = len(xadj) - 1
    src = np.repeat(np.arange(n), np.diff(xadj))
    lo, hi = np.minimum(src, adj), np.maximum(src, adj)
    return (((lo * 7919 + hi * 104729 + seed) % 997) + 1).astype(np.int64)


def _hub(n_leaves=12500, extra=3):
    """A hub joined to n_leaves vertices in runs (chunked: above 10 000), and a
    ring over the leaves."""
    nbrs = [[] for _ in range(n_leaves + 1)]
    hub = n_leaves
    for v in range(n_leaves):
        if v % 7 != 3:  # gaps between runs of consecutive ids
            nbrs[hub].append(v)
            nbrs[v].append(hub)
        w = (v + extra) % n_leaves
        if w != v:
            nbrs[v].append(w)
            nbrs[w].append(v)
    nbrs = [sorted(set(a)) for a in nbrs]
    xadj = np.zeros(len(nbrs) + 1, np.int64)
    np.cumsum([len(a) for a in nbrs], out=xadj[1:])
    return xadj, np.concatenate([np.array(a, np.int32) for a in nbrs])


CASES = [
    ("rgg", lambda: synth.rgg2d(1 << 14, 16.0, 3)),
    ("gnm", lambda: synth.gnm(5000, 30000, 4)),
    ("hub", _hub),
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("intervals", [False, True])
@pytest.mark.parametrize("weights", [False, True])
def test_stream_equals_oracle_and_round_trips(name, make, intervals, weights):
    xadj, adj = make()
    n = len(xadj) - 1
    ew = _sym_weights(xadj, adj, 5) if weights else None
    g = tp.graph_from_csr(xadj, adj, None, ew)
    data, off = g.encode_ex(intervals=intervals, weights=weights)
    want, want_off = oracle.encode_ex(xadj, adj, ew, intervals=intervals)
    assert np.array_equal(data.cpu().numpy(), want), (name, intervals, weights)
    assert np.array_equal(off.cpu().numpy().view(np.uint64), want_off)
    if not intervals and not weights:  # the plain stream the rating kernels read
        zd, zoff = g.compress().export_compressed()
        assert np.array_equal(zd.cpu().numpy(), want)
    back = tp.graph_from_stream_ex(n, data, off, intervals=intervals, weighted=weights)
    bx, ba, _, be = back.export_csr()
    assert np.array_equal(bx.cpu().numpy(), xadj) and np.array_equal(ba.cpu().numpy(), adj)
    if weights:
        assert np.array_equal(be.cpu().numpy(), ew)
    # the oracle decodes the GPU's stream to the same graph
    ox, oa, oe = oracle.decode_ex(n, data.cpu().numpy(), off.cpu().numpy().view(np.uint64),
                                  len(adj), intervals=intervals, weighted=weights)
    assert np.array_equal(ox, xadj) and np.array_equal(oa, adj)


def test_corrupt_streams_are_refused():
    xadj, adj = synth.rgg2d(1 << 12, 12.0, 7)
    n = len(xadj) - 1
    g = tp.graph_from_csr(xadj, adj)
    data, off = g.encode_ex(intervals=True, weights=False)
    host = data.cpu().numpy()
    rng = np.random.default_rng(1)
    refused = 0
    for pos in rng.integers(1, len(host) - 2, size=12):
        bad = host.copy()
        bad[pos] ^= 0x5A
        d = torch.from_numpy(bad).cuda()
        try:
            gg = tp.graph_from_stream_ex(n, d, off, intervals=True)
        except tp.TpError:
            refused += 1
            continue
        bx, ba, _, _ = gg.export_csr()  # a change that still decodes to a valid graph
        assert not (np.array_equal(bx.cpu().numpy(), xadj) and np.array_equal(ba.cpu().numpy(), adj))
    assert refused >= 6
    tp.graph_from_stream_ex(n, data, off, intervals=True)  # the intact stream still decodes


def test_decoded_weighted_graph_partitions_like_the_oracle():
    xadj, adj = synth.gnm(3000, 15000, 9)
    ew = _sym_weights(xadj, adj, 2)
    g = tp.graph_from_csr(xadj, adj, None, ew)
    data, off = g.encode_ex(intervals=True, weights=True)
    back = tp.graph_from_stream_ex(len(xadj) - 1, data, off, intervals=True, weighted=True)
    part, st = tp.partition(back, 8, 0.03, tp.default_params(seed=4))
    want, wst = oracle.partition(oracle.Graph(xadj, adj, None, ew), 8, 0.03, oracle.Params(seed=4))
    assert np.array_equal(part.cpu().numpy(), want) and st["cut"] == wst["cut"]
