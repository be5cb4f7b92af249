"""The last level of the rating order on the GPU: two labels with the same
rating and the same 32-bit tie hash are told apart by the smaller label.

The pair is found by search for the hash key of one vertex; that vertex
gets both labels twice among its neighbours (the top rating), padded with
single-label neighbours to reach each degree tier (lane, small warp, mid
table, global table, chunked hub), in either neighbour order, as CSR and as
compressed graph. Every sub-round is compared with the oracle, vertex by
vertex.
"""
import numpy as np
import pytest

import oracle
from tests import _brute as bf

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2410_19119_gb300 as tp  # noqa: E402

RK = 0x5EED_0F_7135
S = 1  # every vertex active


def _tie_vec(hv, xs):
    z = np.uint64(hv) ^ (xs + np.uint64(bf.GAMMA))
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    return z >> np.uint64(32)


def _colliding_pair(hv, lo=1 << 10, span=1 << 18):
    xs = np.arange(lo, lo + span, dtype=np.uint64)
    t = _tie_vec(hv, xs)
    order = np.argsort(t, kind="stable")
    dup = np.nonzero(t[order][1:] == t[order][:-1])[0]
    assert len(dup) > 0
    x1, x2 = sorted((int(xs[order[dup[0]]]), int(xs[order[dup[0] + 1]])))
    assert bf.tie(hv, x1) == bf.tie(hv, x2)
    return x1, x2


def _star(d):
    """Vertex 0 adjacent to 1..d, nothing else."""
    xadj = np.zeros(d + 2, np.int64)
    xadj[1] = d
    xadj[2:] = d + np.arange(1, d + 1)
    adj = np.concatenate([np.arange(1, d + 1), np.zeros(d)]).astype(np.int32)
    return xadj, adj


@pytest.mark.parametrize("deg", [4, 40, 100, 600, 10500])
@pytest.mark.parametrize("compressed", [False, True])
def test_equal_rating_and_tie_hash_go_to_the_smaller_label(deg, compressed):
    hv = oracle.step(oracle.step(RK, 0), oracle.tag(oracle.TAG_TIE))
    x1, x2 = _colliding_pair(hv)
    xadj, adj = _star(deg)
    n = deg + 1
    og = oracle.Graph(xadj, adj)
    g = tp.graph_from_csr(xadj, adj)
    if compressed:
        g = g.compress()
    for first, second in ((x1, x2), (x2, x1)):
        label = np.zeros(n, np.int32)
        label[0] = 7  # own label, rated 0
        label[1:3] = first
        label[3:5] = second
        label[5:] = x2 + 1 + np.arange(n - 5)  # one neighbour each: rating 1
        nl = int(label.max()) + 1
        lw = np.bincount(label, minlength=nl).astype(np.int64)
        want_l, want_w = label.copy(), lw.copy()
        oracle.lp_subround(og, want_l, want_w, nl, 1 << 20, None, RK, S, 0)
        assert want_l[0] == x1  # the pin the oracle already carries
        dl = torch.from_numpy(label).cuda()
        dw = torch.from_numpy(lw).cuda()
        tp.lp_subround(g, dl, dw, 1 << 20, RK, S, 0)
        assert np.array_equal(dl.cpu().numpy(), want_l), (deg, compressed, first)
        assert np.array_equal(dw.cpu().numpy(), want_w), (deg, compressed, first)
    g.check()
