"""Brute-force restatements of the method's definitions for tiny inputs.

Used only to pin the C oracle: each function enumerates what the definition
quantifies over (every label, every prefix, every assignment) instead of
following the oracle's data structures.
"""
import itertools

import numpy as np

M64 = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15


def mix64(z):
    z &= M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def step(h, x):
    return mix64(h ^ ((x + GAMMA) & M64))


def round_key(seed, tag, a, b):
    return step(step(step(seed, tag), a), b)


def tie(hv, x):
    return step(hv, x) >> 32


def ratings(xadj, adj, ew, u, label, nlabels):
    """R[x] for every label x by a full scan of N(u) per label."""
    R = [0] * nlabels
    for x in range(nlabels):
        for e in range(xadj[u], xadj[u + 1]):
            if label[adj[e]] == x:
                R[x] += int(ew[e])
    return R


def rate(xadj, adj, ew, vw, u, label, lw, nlabels, cap, ignore_cap, hv):
    """(moves, target, gain) for vertex u against the given snapshot."""
    R = ratings(xadj, adj, ew, u, label, nlabels)
    own = int(label[u])
    cands = [x for x in range(nlabels)
             if x != own and R[x] > 0 and (ignore_cap or lw[x] + vw[u] <= cap[x])]
    if not cands:
        return False, -1, 0
    best = min(cands, key=lambda x: (-R[x], tie(hv, x), x))
    if R[best] <= R[own]:
        return False, -1, 0
    return True, best, R[best] - R[own]


def subround(xadj, adj, ew, vw, label, lw, nlabels, cap, rk, S, s, tie_tag):
    """One synchronous sub-round; returns new (label, lw)."""
    n = len(xadj) - 1
    moves = []
    for u in range(n):
        hu = step(rk, u)
        if hu % S != s:
            continue
        ok, t, g = rate(xadj, adj, ew, vw, u, label, lw, nlabels, cap, False, step(hu, tie_tag))
        if ok:
            moves.append((u, t, g))
    approved = []
    for t in sorted({m[1] for m in moves}):
        mv = sorted([m for m in moves if m[1] == t], key=lambda m: (-m[2], m[0]))
        # the longest prefix that fits (searched from the full list downwards)
        for L in range(len(mv), -1, -1):
            if lw[t] + sum(int(vw[m[0]]) for m in mv[:L]) <= cap[t]:
                approved += mv[:L]
                break
    label = label.copy()
    lw = lw.copy()
    for u, t, _ in approved:
        lw[label[u]] -= vw[u]
        lw[t] += vw[u]
        label[u] = t
    return label, lw


def cut(xadj, adj, ew, part):
    c = 0
    for u in range(len(xadj) - 1):
        for e in range(xadj[u], xadj[u + 1]):
            if part[u] != part[adj[e]]:
                c += int(ew[e])
    return c // 2


def dense(xadj, adj, ew):
    n = len(xadj) - 1
    A = np.zeros((n, n), np.int64)
    for u in range(n):
        for e in range(xadj[u], xadj[u + 1]):
            A[u, adj[e]] = ew[e]
    return A


def min_bisection_cut(xadj, adj, ew, vw, cap0, cap1):
    """Smallest cut over all 2-way assignments with side weights within caps."""
    n = len(xadj) - 1
    best = None
    for bits in itertools.product((0, 1), repeat=n):
        w0 = sum(int(vw[u]) for u in range(n) if bits[u] == 0)
        w1 = sum(int(vw[u]) for u in range(n)) - w0
        if w0 > cap0 or w1 > cap1:
            continue
        c = cut(xadj, adj, ew, bits)
        best = c if best is None else min(best, c)
    return best


def rebalance(xadj, adj, ew, vw, part, B, k, l_max):
    part = list(part)
    B = list(B)
    n = len(xadj) - 1
    while True:
        over = [b for b in range(k) if B[b] > l_max]
        if not over:
            return part, B, 0
        b = over[0]
        best = None
        for u in range(n):
            if part[u] != b:
                continue
            R = ratings(xadj, adj, ew, u, part, k)
            feas = [t for t in range(k) if t != b and B[t] + vw[u] <= l_max]
            if not feas:
                continue
            t = min(feas, key=lambda x: (-R[x], x))
            cand = (R[b] - R[t], u, t)
            best = cand if best is None or cand[:2] < best[:2] else best
        if best is None:
            return part, B, 1
        _, u, t = best
        B[b] -= vw[u]
        B[t] += vw[u]
        part[u] = t


def random_graph(rng, n, p, max_w=1):
    """Symmetric random CSR with optional random edge/node weights."""
    edges = {}
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                edges[(u, v)] = int(rng.integers(1, max_w + 1))
    nb = [[] for _ in range(n)]
    for (u, v), w in edges.items():
        nb[u].append((v, w))
        nb[v].append((u, w))
    xadj = [0]
    adj, ew = [], []
    for u in range(n):
        for v, w in sorted(nb[u]):
            adj.append(v)
            ew.append(w)
        xadj.append(len(adj))
    vw = rng.integers(1, max_w + 1, size=n)
    return (np.array(xadj, np.int64), np.array(adj, np.int32), np.array(ew, np.int64),
            np.array(vw, np.int64))
