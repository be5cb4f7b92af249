"""tp_metrics_static: the partition metrics without device allocation.

Callers that cannot allocate device memory when they need the metrics
(services with a device-memory footprint fixed up front, callers without an
allocator of their own) use this entry point; its scratch is a fixed array
inside the library. It must give exactly what the allocating tp_metrics and
the oracle give, call after call, since every call reuses (and must clear)
the same array, and it must not allocate at all. This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402

TP_ERR_INVALID = 1
TP_ERR_BUDGET = 6
STATIC_MAX_BLOCKS = 16383


def _static_metrics(g, part, k, stream=None):
    cut = ctypes.c_int64(-1)
    B = np.full(k, -1, np.int64)
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = tp.lib().tp_metrics_static(g.handle, ctypes.c_void_p(part.data_ptr()), k,
                                    ctypes.byref(cut), ctypes.c_void_p(B.ctypes.data),
                                    ctypes.c_void_p(s.cuda_stream))
    return rc, cut.value, B


def _hub_graph():
    """RGG plus a hub joined to 12 000 of its vertices (above the chunking
    threshold of the compressed format, so the hub is stored in chunks)."""
    xadj, adj = synth.rgg2d(20000, 12.0, 5)
    n = len(xadj) - 1
    hub = n
    leaves = np.arange(0, 12000, dtype=np.int64) * 1 + 0
    nbrs = [list(adj[xadj[u]:xadj[u + 1]]) for u in range(n)]
    for v in leaves:
        nbrs[v].append(hub)
    nbrs.append(list(leaves))
    deg = np.array([len(a) for a in nbrs], np.int64)
    x2 = np.zeros(n + 2, np.int64)
    np.cumsum(deg, out=x2[1:])
    a2 = np.concatenate([np.array(sorted(a), np.int32) for a in nbrs])
    return x2, a2


def _cases():
    """(name, host graph for the oracle, device graphs): unit weights as CSR
    and compressed, a compressed graph with a chunked hub, node and edge
    weights."""
    xadj, adj = synth.rgg2d(50000, 16.0, 7)
    csr = tp.graph_from_csr(xadj, adj)
    yield "rgg", oracle.Graph(xadj, adj), (csr, csr.compress())
    hx, ha = _hub_graph()
    hub = tp.graph_from_csr(hx, ha)
    yield "hub", oracle.Graph(hx, ha), (hub.compress(), hub)
    rng = np.random.default_rng(11)
    wx, wa = synth.gnm(30000, 120000, 3)
    vw = rng.integers(1, 50, size=len(wx) - 1).astype(np.int64)
    ew = np.zeros(len(wa), np.int64)
    for u in range(len(wx) - 1):  # symmetric edge weights
        for e in range(wx[u], wx[u + 1]):
            v = wa[e]
            if u < v:
                w = int(rng.integers(1, 1000))
                ew[e] = w
                f = wx[v] + np.searchsorted(wa[wx[v]:wx[v + 1]], u)
                ew[f] = w
    yield "weighted", oracle.Graph(wx, wa, vw, ew), (tp.graph_from_csr(wx, wa, vw, ew),)


def test_metrics_static_matches_tp_metrics_and_oracle_twice_in_a_row():
    rng = np.random.default_rng(3)
    for name, og, graphs in _cases():
        n = og.n
        for k in (5, 1000, STATIC_MAX_BLOCKS):
            for _ in range(2):  # the second call must not see the first call's sums
                hpart = rng.integers(0, k, size=n).astype(np.int32)
                want_cut = oracle.cut(og, hpart)
                want_B = oracle.block_weights(og, hpart, k)
                part = torch.from_numpy(hpart).cuda()
                for g in graphs:
                    alloc_cut, alloc_B = tp.metrics(g, part, k)
                    rc, cut, B = _static_metrics(g, part, k)
                    assert rc == 0, name
                    assert cut == want_cut == alloc_cut, (name, k)
                    assert np.array_equal(B, want_B), (name, k)
                    assert np.array_equal(B, alloc_B), (name, k)


def test_metrics_static_allocates_nothing():
    """With a counting allocator installed, tp_metrics allocates and
    tp_metrics_static does not."""
    xadj, adj = synth.rgg2d(20000, 16.0, 2)
    counts = {"alloc": 0, "free": 0}

    def alloc(nbytes, stream):
        counts["alloc"] += 1
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)

    def free(ptr, nbytes, stream):
        counts["free"] += 1
        torch.cuda.caching_allocator_delete(ptr)

    g = tp.graph_from_csr(xadj, adj)
    part = torch.from_numpy((np.arange(len(xadj) - 1) % 7).astype(np.int32)).cuda()
    want_cut, want_B = tp.metrics(g, part, 7)  # warm: tier cache built before counting
    tp.set_allocator(alloc, free)
    try:
        for _ in range(3):
            rc, cut, B = _static_metrics(g, part, 7)
            assert rc == 0 and cut == want_cut and np.array_equal(B, want_B)
        assert counts == {"alloc": 0, "free": 0}
        tp.metrics(g, part, 7)
        assert counts["alloc"] > 0 and counts["free"] == counts["alloc"]
    finally:
        tp.use_default_allocator()


def test_metrics_static_rejects_block_ids_out_of_range():
    xadj, adj = synth.gnm(2000, 8000, 4)
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    hpart = (np.arange(2000) % 9).astype(np.int32)
    for bad in (9, -1, STATIC_MAX_BLOCKS + 5):
        p = hpart.copy()
        p[1234] = bad
        rc, _, _ = _static_metrics(g, torch.from_numpy(p).cuda(), 9)
        assert rc == TP_ERR_INVALID
    rc, cut, B = _static_metrics(g, torch.from_numpy(hpart).cuda(), 9)  # still exact afterwards
    assert rc == 0 and cut == oracle.cut(og, hpart)
    assert np.array_equal(B, oracle.block_weights(og, hpart, 9))


def test_metrics_static_rejects_k_beyond_its_scratch():
    xadj, adj = synth.gnm(1000, 4000, 2)
    g = tp.graph_from_csr(xadj, adj)
    part = torch.zeros(1000, dtype=torch.int32, device="cuda")
    rc, _, _ = _static_metrics(g, part, STATIC_MAX_BLOCKS)
    assert rc == 0
    rc, _, _ = _static_metrics(g, part, STATIC_MAX_BLOCKS + 1)
    assert rc == TP_ERR_BUDGET


def test_metrics_static_refuses_a_capturing_stream_without_breaking_the_capture():
    """The call synchronises, so it cannot be captured; on a capturing stream
    it returns an error before enqueuing anything and the capture survives."""
    xadj, adj = synth.gnm(1000, 4000, 2)
    g = tp.graph_from_csr(xadj, adj)
    part = torch.zeros(1000, dtype=torch.int32, device="cuda")
    x = torch.zeros(16, device="cuda")
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=side):
        rc, _, _ = _static_metrics(g, part, 4, stream=side)
        x += 1
    assert rc == TP_ERR_INVALID
    graph.replay()
    torch.cuda.synchronize()
    assert float(x.sum()) == 16.0
