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
        lib.syn_rhg.restype = vp
        lib.syn_rhg.argtypes = [i64, f64, f64, u64]
        lib.syn_rhg_brute.restype = vp
        lib.syn_rhg_brute.argtypes = [i64, f64, f64, u64]
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


def rhg(n: int, avg_deg: float = 16.0, gamma: float = 2.8, seed: int = 1):
    """Threshold random hyperbolic graph, power-law exponent gamma, angle-ordered ids."""
    return _take(_load().syn_rhg(n, avg_deg, gamma, seed))


def rhg_brute(n: int, avg_deg: float = 16.0, gamma: float = 2.8, seed: int = 1):
    """rhg() with every pair tested directly instead of the band search (tests)."""
    return _take(_load().syn_rhg_brute(n, avg_deg, gamma, seed))


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1):
    """R-MAT, symmetrised and deduplicated, self-loops removed."""
    return _take(_load().syn_rmat(scale, edge_factor, a, b, c, seed))


_GAMMA64 = 0x9E3779B97F4A7C15
_MASK64 = (1 << 64) - 1


def _sm64(seed: int, i: int) -> int:
    """Output i of the splitmix64 stream seeded with seed (as in gen.c)."""
    z = (seed + (i + 1) * _GAMMA64) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


BATCH_GENERATORS = ("gnm", "rgg2d", "rhg")
BATCH_KS = (2, 4, 8, 16, 32)


def batch_recipe(count: int = 4096, seed: int = 1, log2_lo: float = 8.0, log2_hi: float = 16.0):
    """The batched workload: graph i has n = round(2^U[log2_lo, log2_hi]) (draw 2i
    of the stream seeded with seed), generator i mod 3 (G(n,m) with average
    degree 8, RGG-2D with average degree 12, RHG with average degree 16 and
    power-law exponent 2.8), k = BATCH_KS[draw 2i+1 mod 5] and graph seed
    (seed << 32) + i. Returns a list of dicts."""
    out = []
    for i in range(count):
        u = (_sm64(seed, 2 * i) >> 11) * (1.0 / 9007199254740992.0)
        n = int(round(2.0 ** (log2_lo + (log2_hi - log2_lo) * u)))
        gen = BATCH_GENERATORS[i % 3]
        k = BATCH_KS[_sm64(seed, 2 * i + 1) % len(BATCH_KS)]
        out.append({"gen": gen, "n": n, "k": k, "seed": (seed << 32) + i,
                    "deg": {"gnm": 8.0, "rgg2d": 12.0, "rhg": 16.0}[gen]})
    return out


def batch_graph(spec):
    """CSR of one batch_recipe entry."""
    n, s = spec["n"], spec["seed"]
    if spec["gen"] == "gnm":
        return gnm(n, int(spec["deg"] * n) // 2, s)
    if spec["gen"] == "rgg2d":
        return rgg2d(n, spec["deg"], s)
    return rhg(n, spec["deg"], 2.8, s)
