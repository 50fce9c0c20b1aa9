"""Small deterministic graph families with known triangle counts.

Each function returns ``(n, src, dst)`` with int32 numpy arrays.  The triangle
counts of these families are textbook facts (they are not stated in the paper)
and are used by the tests to pin the oracle:

=========================  ==========================  =======================
family                      vertices                    triangles
=========================  ==========================  =======================
complete K_n                n                           C(n,3)
complete bipartite K_a,b    a+b                         0
complete tripartite K_a,b,c a+b+c                       a*b*c
wheel W_n (hub + C_{n-1})   n                           n-1 for n >= 5; 4 for n=4
cycle C_n                   n                           1 if n = 3 else 0
path P_n, random tree       n                           0
friendship F_k              2k+1                        k
book K_{1,1,c}              c+2                         c
star + perfect matching     L+1 (L even)                L/2
=========================  ==========================  =======================
"""
from __future__ import annotations

import itertools

import numpy as np


def _pack(n, pairs):
    if len(pairs) == 0:
        return n, np.zeros(0, np.int32), np.zeros(0, np.int32)
    a = np.asarray(pairs, dtype=np.int64)
    return n, a[:, 0].astype(np.int32), a[:, 1].astype(np.int32)


def complete(n):
    return _pack(n, list(itertools.combinations(range(n), 2)))


def complete_bipartite(a, b):
    return _pack(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def complete_tripartite(a, b, c):
    parts = [range(0, a), range(a, a + b), range(a + b, a + b + c)]
    pairs = []
    for p, q in itertools.combinations(parts, 2):
        pairs += [(i, j) for i in p for j in q]
    return _pack(a + b + c, pairs)


def cycle(n):
    return _pack(n, [(i, (i + 1) % n) for i in range(n)])


def path(n):
    return _pack(n, [(i, i + 1) for i in range(n - 1)])


def wheel(n):
    """Hub 0 joined to every vertex of the cycle 1..n-1 (n vertices in total)."""
    rim = n - 1
    pairs = [(0, i) for i in range(1, n)]
    pairs += [(1 + i, 1 + (i + 1) % rim) for i in range(rim)]
    return _pack(n, pairs)


def friendship(k):
    """k triangles sharing the single vertex 0."""
    pairs = []
    for i in range(k):
        a, b = 1 + 2 * i, 2 + 2 * i
        pairs += [(0, a), (0, b), (a, b)]
    return _pack(2 * k + 1, pairs)


def book(c):
    """K_{1,1,c}: the spine edge (0,1) and c pages joined to both ends."""
    pairs = [(0, 1)] + [(0, 2 + i) for i in range(c)] + [(1, 2 + i) for i in range(c)]
    return _pack(c + 2, pairs)


def star_matching(leaves):
    """Hub 0 joined to `leaves` (even) leaves, which are paired by a perfect matching."""
    assert leaves % 2 == 0
    pairs = [(0, 1 + i) for i in range(leaves)]
    pairs += [(1 + 2 * i, 2 + 2 * i) for i in range(leaves // 2)]
    return _pack(leaves + 1, pairs)


def random_tree(n, seed):
    """Uniform random labelled tree from a random Pruefer sequence (numpy RNG)."""
    if n <= 1:
        return _pack(n, [])
    if n == 2:
        return _pack(2, [(0, 1)])
    rng = np.random.default_rng(seed)
    seq = rng.integers(0, n, size=n - 2)
    degree = np.ones(n, dtype=np.int64)
    for x in seq:
        degree[x] += 1
    pairs = []
    import heapq
    leaves = [i for i in range(n) if degree[i] == 1]
    heapq.heapify(leaves)
    for x in seq:
        leaf = heapq.heappop(leaves)
        pairs.append((leaf, int(x)))
        degree[x] -= 1
        if degree[x] == 1:
            heapq.heappush(leaves, int(x))
    u, v = heapq.heappop(leaves), heapq.heappop(leaves)
    pairs.append((u, v))
    return _pack(n, pairs)


def disjoint_union(*graphs):
    """Disjoint union of (n, src, dst) graphs; vertex ids are shifted block by block."""
    n_tot, srcs, dsts = 0, [], []
    for n, s, d in graphs:
        srcs.append(s.astype(np.int64) + n_tot)
        dsts.append(d.astype(np.int64) + n_tot)
        n_tot += n
    if not srcs:
        return 0, np.zeros(0, np.int32), np.zeros(0, np.int32)
    return n_tot, np.concatenate(srcs).astype(np.int32), np.concatenate(dsts).astype(np.int32)


def random_graph(n, p, seed):
    """Small G(n, p) from numpy's RNG (each pair kept with probability p)."""
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(n, 1)
    keep = rng.random(len(iu[0])) < p
    return n, iu[0][keep].astype(np.int32), iu[1][keep].astype(np.int32)
