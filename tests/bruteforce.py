"""Independent reference computations used to pin the oracle.

Nothing here calls the oracle or the CUDA path.  These are the plain
definitions of Sec. II of the paper written with numpy:

* a triangle is a set {u, v, w} whose three pairs are all edges;
* T_v is the number of edges among the neighbours of v;
* for a simple graph with adjacency matrix A, trace(A^3) = 6 T and
  (A^3)_vv = 2 T_v.
"""
import itertools

import numpy as np


def adjacency(n, src, dst):
    """Dense boolean adjacency of the simple graph (self-loops dropped, repeats merged)."""
    A = np.zeros((n, n), dtype=bool)
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    A[src[keep], dst[keep]] = True
    A[dst[keep], src[keep]] = True
    return A


def triangles_by_triples(n, src, dst):
    """Check every triple (u < v < w): the naive algorithm of Sec. III-A."""
    A = adjacency(n, src, dst)
    t = 0
    for u, v, w in itertools.combinations(range(n), 3):
        if A[u, v] and A[v, w] and A[u, w]:
            t += 1
    return t


def triangle_list(n, src, dst):
    """All triangles as sorted triples, by a vectorised triple check."""
    A = adjacency(n, src, dst)
    out = []
    for u in range(n):
        for v in np.nonzero(A[u, u + 1:])[0] + u + 1:
            ws = np.nonzero(A[u, v + 1:] & A[v, v + 1:])[0] + v + 1
            out.extend((u, int(v), int(w)) for w in ws)
    return out


def triangles_fast(n, src, dst):
    """Vectorised triple check for n up to a few hundred."""
    return len(triangle_list(n, src, dst))


def trace_a3(n, src, dst):
    """(trace(A^3) / 6, diag(A^3) / 2) with exact int64 matrix products."""
    A = adjacency(n, src, dst).astype(np.int64)
    A2 = A @ A
    diag = np.einsum("ij,ji->i", A2, A)
    assert int(diag.sum()) % 6 == 0
    return int(diag.sum()) // 6, diag // 2


def per_vertex_by_definition(n, src, dst):
    """T_v = number of edges among the neighbours of v (Sec. II)."""
    A = adjacency(n, src, dst)
    tv = np.zeros(n, dtype=np.int64)
    for v in range(n):
        nb = np.nonzero(A[v])[0]
        sub = A[np.ix_(nb, nb)]
        tv[v] = int(sub.sum()) // 2
    return tv
