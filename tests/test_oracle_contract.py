"""Pins for the oracle's contraction (Section "Contraction"): the coarse graph
equals P^T A P with the diagonal removed, weights are preserved, and the
identity / all-in-one clusterings reduce to the input / a single vertex."""
import numpy as np
import pytest

import oracle
import synth
from tests import _brute as bf


def _check(xadj, adj, ew, vw, C):
    g = oracle.Graph(xadj, adj, vw, ew)
    cg, mp = oracle.contract(g, C)
    labels = np.unique(C)
    assert cg.n == len(labels)
    # coarse ids are the ranks of the labels
    assert np.array_equal(mp, np.searchsorted(labels, C))
    # node weights
    assert np.array_equal(cg.vw, np.bincount(mp, weights=vw, minlength=cg.n).astype(np.int64))
    # canonical CSR: sorted, no self-loops, symmetric
    assert oracle.validate(cg) == 0
    # A' = P^T A P without the diagonal (dense check for small graphs)
    if len(xadj) <= 400:
        A = bf.dense(xadj, adj, ew)
        P = np.zeros((len(xadj) - 1, cg.n), np.int64)
        P[np.arange(len(xadj) - 1), mp] = 1
        Ac = P.T @ A @ P
        np.fill_diagonal(Ac, 0)
        assert np.array_equal(Ac, bf.dense(cg.xadj, cg.adj, cg.ew))
    # total coarse edge weight == fine inter-cluster weight
    src = np.repeat(np.arange(len(xadj) - 1), np.diff(xadj))
    inter = C[src] != C[adj]
    assert cg.ew.sum() == ew[inter].sum()
    return cg, mp


@pytest.mark.parametrize("seed", range(6))
def test_contract_dense_equivalence(seed):
    rng = np.random.default_rng(seed)
    xadj, adj, ew, vw = bf.random_graph(rng, 30, 0.2, 5)
    C = rng.integers(0, 30, size=30).astype(np.int32)
    _check(xadj, adj, ew, vw, C)


def test_contract_identity_and_all_in_one():
    xadj, adj = synth.gnm(300, 1500, 4)
    n = len(xadj) - 1
    ew = np.arange(1, len(adj) + 1, dtype=np.int64)
    # symmetric weights: w(u,v) = w(v,u) = min index of the two entries
    src = np.repeat(np.arange(n), np.diff(xadj))
    key = np.minimum(src, adj).astype(np.int64) * n + np.maximum(src, adj)
    ew = (key % 97 + 1).astype(np.int64)
    vw = (np.arange(n) % 5 + 1).astype(np.int64)
    cg, mp = _check(xadj, adj, ew, vw, np.arange(n, dtype=np.int32))
    assert np.array_equal(cg.xadj, xadj) and np.array_equal(cg.adj, adj)
    assert np.array_equal(cg.ew, ew) and np.array_equal(cg.vw, vw)
    cg, mp = _check(xadj, adj, ew, vw, np.full(n, 17, np.int32))
    assert cg.n == 1 and cg.m2 == 0 and cg.vw[0] == vw.sum()


def test_contract_after_clustering_large():
    xadj, adj = synth.rgg2d(20000, 16.0, 2)
    g = oracle.Graph(xadj, adj)
    C = oracle.cluster(g, 40, oracle.Params(), 0)
    ones = np.ones(len(adj), np.int64)
    _check(xadj, adj, ones, np.ones(len(xadj) - 1, np.int64), C)


def test_validate_names_each_broken_rule():
    # the validator the contraction pins rely on: every rule of the graph
    # representation, broken one at a time on a valid 4-cycle with weights
    xadj = np.array([0, 2, 4, 6, 8], np.int64)
    adj = np.array([1, 3, 0, 2, 1, 3, 0, 2], np.int32)
    ew = np.array([5, 7, 5, 6, 6, 4, 7, 4], np.int64)
    vw = np.array([1, 2, 3, 4], np.int64)
    assert oracle.validate(oracle.Graph(xadj, adj, vw, ew)) == 0

    def code(xadj=xadj, adj=adj, ew=ew, vw=vw):
        return oracle.validate(oracle.Graph(xadj, adj, vw, ew))

    assert code(xadj=np.array([1, 2, 4, 6, 8], np.int64)) == 1  # does not start at 0
    # codes name the first broken rule in vertex order: break each at vertex 0
    assert code(xadj=np.array([0, -1, 4, 6, 8], np.int64)) == 2  # offsets decrease
    assert code(vw=np.array([1, 0, 3, 4], np.int64)) == 3  # node weight not positive
    bad = adj.copy()
    bad[0] = 9
    assert code(adj=bad) == 4  # neighbour id out of range
    bad = adj.copy()
    bad[0] = 0
    assert code(adj=bad) == 5  # self-loop
    bad, badw = adj.copy(), ew.copy()
    bad[0], bad[1] = bad[1], bad[0]
    badw[0], badw[1] = badw[1], badw[0]
    assert code(adj=bad, ew=badw) == 6  # unsorted neighbourhood
    bad = ew.copy()
    bad[1] = 0
    assert code(ew=bad) == 7  # edge weight not positive
    bad = ew.copy()
    bad[1] = 8
    assert code(ew=bad) == 8  # w(0,3) != w(3,0)
    # an edge stored in one direction only: 0-2 added at vertex 0 alone
    x2 = np.array([0, 3, 5, 7, 9], np.int64)
    a2 = np.array([1, 2, 3, 0, 2, 1, 3, 0, 2], np.int32)
    w2 = np.array([5, 1, 7, 5, 6, 6, 4, 7, 4], np.int64)
    assert code(xadj=x2, adj=a2, ew=w2) == 8
