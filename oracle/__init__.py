"""Sequential CPU oracle of the deterministic multilevel partitioner.

TEST INFRASTRUCTURE ONLY. The product path never imports this package: only
tests/, the smoke check and the CPU-baseline / reference legs of bench.py do.
It wraps the plain C implementation in this directory (see oracle.h for which
passage of the paper each function restates and how each is pinned).
"""
import ctypes
import math
import os

import numpy as np

from .build import LIB, build

_lib = None
i64, i32, u64, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_void_p


class _CGraph(ctypes.Structure):
    _fields_ = [("n", i64), ("m2", i64), ("xadj", vp), ("adj", vp), ("vw", vp), ("ew", vp)]


class _CParams(ctypes.Structure):
    _fields_ = [("seed", u64), ("cluster_rounds", i32), ("refine_rounds", i32),
                ("sub_rounds", i32), ("c_lim", i32), ("ip_attempts", i32), ("two_hop", i32),
                ("max_levels", i32), ("fm_passes", i32)]


class _CStats(ctypes.Structure):
    _fields_ = [("cut", i64), ("max_block_weight", i64), ("l_max", i64), ("u_max", i64),
                ("imbalance", ctypes.c_double), ("levels", i32), ("balanced", i32),
                ("level_n", i64 * 64), ("level_m2", i64 * 64)]


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        lib = ctypes.CDLL(LIB)
        sig = {
            "orc_mix64": (u64, [u64]),
            "orc_step": (u64, [u64, u64]),
            "orc_round_key": (u64, [u64, u64, u64, u64]),
            "orc_tag": (u64, [ctypes.c_int]),
            "orc_varint_len": (ctypes.c_int, [u64]),
            "orc_varint_put": (ctypes.c_int, [vp, u64]),
            "orc_encoded_size": (i64, [i64, vp, vp]),
            "orc_encode": (i64, [i64, vp, vp, vp, vp]),
            "orc_decode": (ctypes.c_int, [i64, vp, i64, vp, vp, vp, i64]),
            "orc_encode_ex": (i64, [i64, vp, vp, vp, ctypes.c_int, vp, vp]),
            "orc_fm_refine": (i64, [vp, vp, vp, ctypes.c_int32, i64, ctypes.c_int32]),
            "orc_gt_build": (vp, [vp, vp, ctypes.c_int32]),
            "orc_gt_get": (i64, [vp, i64, ctypes.c_int32]),
            "orc_gt_move": (None, [vp, vp, i64, ctypes.c_int32, ctypes.c_int32]),
            "orc_gt_bytes": (i64, [vp]),
            "orc_gt_layout": (None, [vp, i64, vp, vp, vp, vp]),
            "orc_gt_check": (ctypes.c_int, [vp]),
            "orc_gt_free": (None, [vp]),
            "orc_decode_ex": (ctypes.c_int, [i64, vp, i64, vp, ctypes.c_int, ctypes.c_int, vp, vp,
                                             vp, i64]),
            "orc_rate_vertex": (ctypes.c_int, [vp, i64, vp, vp, i64, vp, ctypes.c_int, u64, vp, vp]),
            "orc_rate_vertex_sorted": (ctypes.c_int, [vp, i64, vp, vp, i64, vp, ctypes.c_int, u64, vp, vp]),
            "orc_lp_subround": (i64, [vp, vp, vp, i64, i64, vp, u64, i32, i32]),
            "orc_lp_rounds": (i64, [vp, vp, vp, i64, i64, vp, u64, u64, u64, u64, i32, i32]),
            "orc_two_hop": (None, [vp, vp, vp, i64, u64, i64]),
            "orc_cluster": (None, [vp, i64, vp, i64, vp]),
            "orc_contract": (i64, [vp, vp, vp, vp]),
            "orc_graph_free": (None, [vp]),
            "orc_initial_partition": (None, [vp, i32, i64, vp, vp]),
            "orc_block_weights": (None, [vp, vp, i32, vp]),
            "orc_cut": (i64, [vp, vp]),
            "orc_rebalance": (ctypes.c_int, [vp, vp, vp, i32, i64]),
            "orc_refine": (i64, [vp, vp, vp, i32, i64, vp, i64]),
            "orc_cluster_cap": (i64, [i64, i32, i64]),
            "orc_block_cap": (i64, [i64, i32, i64]),
            "orc_validate": (ctypes.c_int, [vp]),
            "orc_partition": (ctypes.c_int, [vp, i32, i64, vp, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data if a is not None else None


class Graph:
    """CSR graph held in numpy arrays (int64 xadj, int32 adj, int64 weights)."""

    def __init__(self, xadj, adj, vw=None, ew=None, implicit_unit=False):
        """implicit_unit: no weight arrays at all (unit weights, read as 1 by every
        function; large graphs need not carry arrays of ones)."""
        self.xadj = np.ascontiguousarray(xadj, dtype=np.int64)
        self.adj = np.ascontiguousarray(adj, dtype=np.int32)
        n = len(self.xadj) - 1
        if implicit_unit:
            self.vw = self.ew = None
        else:
            self.vw = np.ones(n, np.int64) if vw is None else np.ascontiguousarray(vw, dtype=np.int64)
            self.ew = np.ones(len(self.adj), np.int64) if ew is None else np.ascontiguousarray(ew, dtype=np.int64)
        self._c = _CGraph(n, len(self.adj), _p(self.xadj), _p(self.adj), _p(self.vw), _p(self.ew))

    @property
    def n(self):
        return len(self.xadj) - 1

    @property
    def m2(self):
        return len(self.adj)

    @property
    def c(self):
        return ctypes.byref(self._c)


class Params:
    def __init__(self, seed=1, cluster_rounds=5, refine_rounds=5, sub_rounds=8, c_lim=160,
                 ip_attempts=8, two_hop=1, max_levels=64, fm_passes=0):
        self.seed, self.cluster_rounds, self.refine_rounds = seed, cluster_rounds, refine_rounds
        self.sub_rounds, self.c_lim, self.ip_attempts = sub_rounds, c_lim, ip_attempts
        self.two_hop, self.max_levels, self.fm_passes = two_hop, max_levels, fm_passes

    @property
    def c(self):
        return ctypes.byref(_CParams(self.seed, self.cluster_rounds, self.refine_rounds,
                                     self.sub_rounds, self.c_lim, self.ip_attempts,
                                     self.two_hop, self.max_levels, self.fm_passes))


def eps_to_ppm(eps: float) -> int:
    """eps as integer parts per million, rounded half away from zero (llround)."""
    return int(math.floor(eps * 1e6 + 0.5))


# ---------------------------------------------------------------- hashing
def mix64(z):
    return _load().orc_mix64(z & (2**64 - 1))


def step(h, x):
    return _load().orc_step(h & (2**64 - 1), x & (2**64 - 1))


def round_key(seed, tag, a, b):
    return _load().orc_round_key(seed, tag, a & (2**64 - 1), b & (2**64 - 1))


TAG_CLUSTER, TAG_REFINE, TAG_TWOHOP, TAG_IPSEED, TAG_IPLP, TAG_TIE = range(6)


def tag(which):
    return _load().orc_tag(which)


# ---------------------------------------------------------------- codec
def varint(x: int) -> bytes:
    buf = np.zeros(16, np.uint8)
    k = _load().orc_varint_put(buf.ctypes.data, x)
    return bytes(buf[:k])


def encoded_size(xadj, adj):
    xadj = np.ascontiguousarray(xadj, np.int64)
    adj = np.ascontiguousarray(adj, np.int32)
    return _load().orc_encoded_size(len(xadj) - 1, xadj.ctypes.data, adj.ctypes.data)


def encode(xadj, adj):
    """Returns (bytes uint8[nbytes], off uint64[n+1])."""
    xadj = np.ascontiguousarray(xadj, np.int64)
    adj = np.ascontiguousarray(adj, np.int32)
    n = len(xadj) - 1
    size = encoded_size(xadj, adj)
    out = np.zeros(size, np.uint8)
    off = np.zeros(n + 1, np.uint64)
    got = _load().orc_encode(n, xadj.ctypes.data, adj.ctypes.data, out.ctypes.data, off.ctypes.data)
    assert got == size
    return out, off


def decode(n, data, off, m2_cap):
    data = np.ascontiguousarray(data, np.uint8)
    off = np.ascontiguousarray(off, np.uint64)
    xadj = np.zeros(n + 1, np.int64)
    adj = np.zeros(max(m2_cap, 1), np.int32)
    r = _load().orc_decode(n, data.ctypes.data, len(data), off.ctypes.data, xadj.ctypes.data,
                           adj.ctypes.data, m2_cap)
    if r != 0:
        raise ValueError("corrupt compressed graph")
    return xadj, adj[: xadj[n]]


def encode_ex(xadj, adj, ew=None, intervals=True):
    """Interval + weight format: returns (bytes uint8[nbytes], off uint64[n+1])."""
    xadj = np.ascontiguousarray(xadj, np.int64)
    adj = np.ascontiguousarray(adj, np.int32)
    ewp = None
    if ew is not None:
        ew = np.ascontiguousarray(ew, np.int64)
        ewp = ew.ctypes.data
    n = len(xadj) - 1
    lib = _load()
    size = lib.orc_encode_ex(n, xadj.ctypes.data, adj.ctypes.data, ewp, int(intervals), None, None)
    out = np.zeros(max(size, 1), np.uint8)
    off = np.zeros(n + 1, np.uint64)
    got = lib.orc_encode_ex(n, xadj.ctypes.data, adj.ctypes.data, ewp, int(intervals),
                            out.ctypes.data, off.ctypes.data)
    assert got == size
    return out[:size], off


def decode_ex(n, data, off, m2_cap, intervals=True, weighted=False):
    """Returns (xadj, adj, ew) of an interval + weight stream (ew all ones
    when the stream holds no weights)."""
    data = np.ascontiguousarray(data, np.uint8)
    off = np.ascontiguousarray(off, np.uint64)
    xadj = np.zeros(n + 1, np.int64)
    adj = np.zeros(max(m2_cap, 1), np.int32)
    ew = np.ones(max(m2_cap, 1), np.int64)
    r = _load().orc_decode_ex(n, data.ctypes.data, len(data), off.ctypes.data, int(intervals),
                              int(weighted), xadj.ctypes.data, adj.ctypes.data, ew.ctypes.data,
                              m2_cap)
    if r != 0:
        raise ValueError("corrupt compressed graph")
    return xadj, adj[: xadj[n]], ew[: xadj[n]]


def fm_refine(g: "Graph", part, B, k, l_max, passes=8):
    """k-way FM over the gain table, in place on part (int32) and B (int64);
    returns the cut reduction."""
    return _load().orc_fm_refine(g.c, part.ctypes.data, B.ctypes.data, k, l_max, passes)


class GainTable:
    """Space-efficient gain table of a partition (affinity of every vertex to
    every block; dense k values above degree k, sparse hash tables below)."""

    def __init__(self, g: "Graph", part, k):
        self._g = g
        self._part = np.ascontiguousarray(part, np.int32)
        self.k = k
        self._h = _load().orc_gt_build(g.c, self._part.ctypes.data, k)

    def get(self, v, b):
        return _load().orc_gt_get(self._h, v, b)

    def move(self, u, frm, to):
        _load().orc_gt_move(self._h, self._g.c, u, frm, to)

    def bytes(self):
        return _load().orc_gt_bytes(self._h)

    def layout(self, v):
        cap, st = ctypes.c_int64(), ctypes.c_int64()
        w, d = ctypes.c_int32(), ctypes.c_int32()
        _load().orc_gt_layout(self._h, v, ctypes.byref(cap), ctypes.byref(w), ctypes.byref(d),
                              ctypes.byref(st))
        return {"cap": cap.value, "width": w.value, "dense": bool(d.value), "stored": st.value}

    def check(self):
        return _load().orc_gt_check(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            _load().orc_gt_free(self._h)
            self._h = None


# ---------------------------------------------------------------- LP
def rate_vertex(g: Graph, u, label, lw, cap_uniform, cap=None, ignore_cap=False, hv=0):
    t = ctypes.c_int32(0)
    gain = ctypes.c_int64(0)
    moved = _load().orc_rate_vertex(g.c, u, label.ctypes.data, lw.ctypes.data, cap_uniform,
                                    _p(cap), int(ignore_cap), hv, ctypes.byref(t), ctypes.byref(gain))
    return bool(moved), t.value, gain.value


def rate_vertex_sorted(g: Graph, u, label, lw, cap_uniform, cap=None, ignore_cap=False, hv=0):
    """rate_vertex for one vertex of a large graph (sort-based ratings)."""
    t = ctypes.c_int32(0)
    gain = ctypes.c_int64(0)
    moved = _load().orc_rate_vertex_sorted(g.c, u, label.ctypes.data, lw.ctypes.data, cap_uniform,
                                           _p(cap), int(ignore_cap), hv, ctypes.byref(t),
                                           ctypes.byref(gain))
    return bool(moved), t.value, gain.value


def vertex_hashes(rk, u):
    """(sub-round hash, tie key) of vertex u under round key rk."""
    hu = step(rk, u)
    return hu, step(hu, tag(TAG_TIE))


def lp_subround(g: Graph, label, lw, nlabels, cap_uniform, cap, rk, S, s):
    """In place on label (int32) and lw (int64); returns the number of moves."""
    return _load().orc_lp_subround(g.c, label.ctypes.data, lw.ctypes.data, nlabels, cap_uniform,
                                   _p(cap), rk, S, s)


def lp_rounds(g: Graph, label, lw, nlabels, cap_uniform, cap, seed, tag_value, a, b0, rounds, S):
    return _load().orc_lp_rounds(g.c, label.ctypes.data, lw.ctypes.data, nlabels, cap_uniform,
                                 _p(cap), seed, tag_value, a, b0, rounds, S)


def two_hop(g: Graph, C, Wc, U, seed, level):
    _load().orc_two_hop(g.c, C.ctypes.data, Wc.ctypes.data, U, seed, level)


def cluster(g: Graph, U, p: Params, level):
    C = np.zeros(max(g.n, 1), np.int32)
    _load().orc_cluster(g.c, U, p.c, level, C.ctypes.data)
    return C[: g.n]


def contract(g: Graph, C):
    """Returns (coarse Graph, map int32[n])."""
    C = np.ascontiguousarray(C, np.int32)
    out = _CGraph()
    mp = np.zeros(max(g.n, 1), np.int32)
    lib = _load()
    nc = lib.orc_contract(g.c, C.ctypes.data, ctypes.byref(out), mp.ctypes.data)
    m2 = out.m2

    def take(ptr, count, dt):
        if count == 0:
            return np.zeros(0, dt)
        return np.ctypeslib.as_array(ctypes.cast(ptr, ctypes.POINTER(np.ctypeslib.as_ctypes_type(dt))),
                                     shape=(count,)).copy()

    coarse = Graph(take(out.xadj, nc + 1, np.int64), take(out.adj, m2, np.int32),
                   take(out.vw, nc, np.int64), take(out.ew, m2, np.int64))
    lib.orc_graph_free(ctypes.byref(out))
    return coarse, mp[: g.n]


# ---------------------------------------------------------------- partitioning
def cluster_cap(W, k, eps_ppm):
    return _load().orc_cluster_cap(W, k, eps_ppm)


def block_cap(W, k, eps_ppm):
    return _load().orc_block_cap(W, k, eps_ppm)


def validate(g: Graph):
    return _load().orc_validate(g.c)


def initial_partition(g: Graph, k, l_max, p: Params):
    part = np.zeros(max(g.n, 1), np.int32)
    _load().orc_initial_partition(g.c, k, l_max, p.c, part.ctypes.data)
    return part[: g.n]


def block_weights(g: Graph, part, k):
    B = np.zeros(k, np.int64)
    _load().orc_block_weights(g.c, np.ascontiguousarray(part, np.int32).ctypes.data, k, B.ctypes.data)
    return B


def cut(g: Graph, part):
    return _load().orc_cut(g.c, np.ascontiguousarray(part, np.int32).ctypes.data)


def rebalance(g: Graph, part, B, k, l_max):
    return _load().orc_rebalance(g.c, part.ctypes.data, B.ctypes.data, k, l_max)


def refine(g: Graph, part, B, k, l_max, p: Params, level):
    return _load().orc_refine(g.c, part.ctypes.data, B.ctypes.data, k, l_max, p.c, level)


def partition(g: Graph, k, eps, p: Params):
    """Returns (part int32[n], stats dict)."""
    part = np.zeros(max(g.n, 1), np.int32)
    st = _CStats()
    r = _load().orc_partition(g.c, k, eps_to_ppm(eps), p.c, part.ctypes.data, ctypes.byref(st))
    if r != 0:
        raise ValueError("invalid partition arguments")
    stats = {
        "cut": st.cut, "max_block_weight": st.max_block_weight, "l_max": st.l_max,
        "u_max": st.u_max, "imbalance": st.imbalance, "levels": st.levels,
        "balanced": bool(st.balanced),
        "level_n": list(st.level_n[: st.levels]), "level_m2": list(st.level_m2[: st.levels]),
    }
    return part[: g.n], stats
