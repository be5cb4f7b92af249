"""Seeded synthetic graphs shaped like the paper's workloads.

This module holds input generation only (no partitioning arithmetic); it feeds
the GPU path and the CPU oracle the same CSR arrays. See gen.c for the exact
definition of each generator.
"""
import ctypes
import os

import numpy as np

from .build import LIB, build

_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            build()
        lib = ctypes.CDLL(LIB)
        vp, i64, i32, u64, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_double
        lib.syn_gnm.restype = vp
        lib.syn_gnm.argtypes = [i64, i64, u64]
        lib.syn_rgg2d.restype = vp
        lib.syn_rgg2d.argtypes = [i64, f64, u64]
        lib.syn_rmat.restype = vp
        lib.syn_rmat.argtypes = [i32, i64, f64, f64, f64, u64]
        lib.syn_n.restype = i64
        lib.syn_n.argtypes = [vp]
        lib.syn_m2.restype = i64
        lib.syn_m2.argtypes = [vp]
        lib.syn_copy.argtypes = [vp, vp, vp]
        lib.syn_free.argtypes = [vp]
        _lib = lib
    return _lib


def _take(h):
    lib = _load()
    n, m2 = lib.syn_n(h), lib.syn_m2(h)
    xadj = np.empty(n + 1, dtype=np.int64)
    adj = np.empty(max(m2, 1), dtype=np.int32)
    lib.syn_copy(h, xadj.ctypes.data, adj.ctypes.data)
    lib.syn_free(h)
    return xadj, adj[:m2]


def gnm(n: int, m: int, seed: int = 1):
    """Uniform G(n,m): m distinct undirected pairs, no self-loops."""
    return _take(_load().syn_gnm(n, m, seed))


def rgg2d(n: int, avg_deg: float = 16.0, seed: int = 1):
    """2D random geometric graph in the unit square, grid-cell vertex order."""
    return _take(_load().syn_rgg2d(n, avg_deg, seed))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1):
    """R-MAT, symmetrised and deduplicated, self-loops removed."""
    return _take(_load().syn_rmat(scale, edge_factor, a, b, c, seed))
