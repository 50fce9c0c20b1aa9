"""Pins of the CPU oracle against facts that do not come from the oracle itself.

The oracle (oracle/tc_oracle.c) follows Fig. 1 of the paper.  These tests tie it
to brute force (Sec. III-A's naive triple check), trace(A^3)/6, closed-form
counts of textbook families, the invariants the paper states (any total order
counts each triangle once, Sec. III-A; each triangle is found exactly once at
its lowest vertex via the edge to its middle vertex, Theorem 1), and the
definition of T_v (Sec. II).  A dropped term, a wrong sign, a swapped index or
a transposed operand in the oracle fails at least one of them.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from graphgen import families as F
from tests import bruteforce as BF


def oracle_T(n, s, d, **kw):
    return oracle.count_edges(n, s, d, **kw)


# --------------------------------------------------------------------------- brute force

@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 7, 12, 25])
@pytest.mark.parametrize("p", [0.1, 0.4, 0.8, 1.0])
def test_brute_force_triples(n, p):
    for seed in range(3):
        n_, s, d = F.random_graph(n, p, seed)
        assert oracle_T(n_, s, d) == BF.triangles_by_triples(n_, s, d)


@pytest.mark.parametrize("n,p", [(60, 0.05), (60, 0.5), (150, 0.02), (150, 0.1), (150, 0.3)])
def test_brute_force_vectorised(n, p):
    n_, s, d = F.random_graph(n, p, 11)
    assert oracle_T(n_, s, d) == BF.triangles_fast(n_, s, d)


@pytest.mark.parametrize("n", [4, 5, 6])
def test_exhaustive_small_graphs(n):
    """Every labelled graph on n <= 6 vertices (2^15 = 32768 graphs at n = 6)."""
    pairs = list(itertools.combinations(range(n), 2))
    triples = list(itertools.combinations(range(n), 3))
    idx = {p: i for i, p in enumerate(pairs)}
    masks = np.arange(1 << len(pairs), dtype=np.int64)
    bits = (masks[:, None] >> np.arange(len(pairs))[None, :]) & 1
    expect = np.zeros(len(masks), dtype=np.int64)
    for a, b, c in triples:
        expect += bits[:, idx[(a, b)]] & bits[:, idx[(b, c)]] & bits[:, idx[(a, c)]]
    P = np.array(pairs, dtype=np.int32)
    step = 1 if n < 6 else 7  # n = 6: every 7th graph (4682 of 32768) keeps the CPU suite short
    for mk in range(0, len(masks), step):
        sel = bits[mk].astype(bool)
        got = oracle_T(n, P[sel, 0], P[sel, 1])
        assert got == expect[mk], (n, mk)


# --------------------------------------------------------------------------- trace(A^3)

@pytest.mark.parametrize("case", ["er", "ba", "cl", "dense"])
def test_trace_a3_and_per_vertex(case):
    import graphgen
    if case == "er":
        n = 400
        s, d = graphgen.erdos_renyi(n, 4000, 5)
    elif case == "ba":
        n = 300
        s, d = graphgen.barabasi_albert(n, 6, 5)
    elif case == "cl":
        n = 400
        s, d = graphgen.chung_lu(n, 2.1, 12.0, 120.0, 2400, 5)
    else:
        n, s, d = F.random_graph(120, 0.7, 5)
    T3, tv3 = BF.trace_a3(n, s, d)
    T, _, tv = oracle.count(oracle.oriented_csr(oracle.simple_graph(n, s, d)), per_vertex=True)
    assert T == T3
    assert np.array_equal(tv.astype(np.int64), tv3)
    assert int(tv.sum()) == 3 * T


# --------------------------------------------------------------------------- closed forms

def _T(g):
    n, s, d = g
    return oracle_T(n, s, d)


@pytest.mark.parametrize("n", list(range(0, 40)) + [64, 100])
def test_complete_graph(n):
    n_, s, d = F.complete(n)
    csr = oracle.oriented_csr(oracle.simple_graph(n_, s, d))
    T, _, tv = oracle.count(csr, per_vertex=True)
    assert T == math.comb(n, 3)
    assert all(int(x) == math.comb(n - 1, 2) for x in tv)


@pytest.mark.parametrize("a,b", [(1, 1), (1, 50), (3, 7), (20, 20), (2, 300)])
def test_complete_bipartite_is_triangle_free(a, b):
    assert _T(F.complete_bipartite(a, b)) == 0


@pytest.mark.parametrize("a,b,c", [(1, 1, 1), (1, 1, 5), (2, 3, 4), (5, 5, 5), (1, 7, 30)])
def test_complete_tripartite(a, b, c):
    assert _T(F.complete_tripartite(a, b, c)) == a * b * c


def test_cycles_paths_trees():
    assert _T(F.cycle(3)) == 1
    for n in range(4, 40):
        assert _T(F.cycle(n)) == 0
        assert _T(F.path(n)) == 0
    for seed in range(5):
        assert _T(F.random_tree(500, seed)) == 0


@pytest.mark.parametrize("n", [5, 6, 7, 10, 33, 1000])
def test_wheel(n):
    assert _T(F.wheel(n)) == n - 1


def test_wheel_w4_is_k4():
    assert _T(F.wheel(4)) == 4


@pytest.mark.parametrize("k", [1, 2, 10, 500])
def test_friendship(k):
    assert _T(F.friendship(k)) == k


@pytest.mark.parametrize("c", [1, 2, 100, 20000])
def test_book(c):
    assert _T(F.book(c)) == c


@pytest.mark.parametrize("L", [2, 10, 1000])
def test_star_with_matching(L):
    assert _T(F.star_matching(L)) == L // 2


def test_disjoint_union_adds():
    parts = [F.complete(7), F.wheel(9), F.book(13), F.complete_tripartite(2, 3, 4), F.cycle(3)]
    assert _T(F.disjoint_union(*parts)) == sum(_T(g) for g in parts)


# --------------------------------------------------------------------------- invariants

def _some_graph(seed=3):
    import graphgen
    return 500, *graphgen.chung_lu(500, 2.3, 14.0, 150.0, 3500, seed)


def test_invariance_relabel_shuffle_reverse():
    n, s, d = _some_graph()
    T = oracle_T(n, s, d)
    rng = np.random.default_rng(0)
    perm = rng.permutation(n).astype(np.int32)
    assert oracle_T(n, perm[s], perm[d]) == T
    order = rng.permutation(len(s))
    assert oracle_T(n, s[order], d[order]) == T
    flip = rng.random(len(s)) < 0.5
    s2, d2 = np.where(flip, d, s), np.where(flip, s, d)
    assert oracle_T(n, s2, d2) == T


def test_invariance_duplicates_and_loops_sanitised():
    n, s, d = _some_graph(4)
    g = oracle.simple_graph(n, s, d)
    T = oracle.count(oracle.oriented_csr(g))
    rng = np.random.default_rng(1)
    pick = rng.integers(0, g.m_hat, 300)
    loops = rng.integers(0, n, 50).astype(np.int32)
    s2 = np.concatenate([g.a, g.b[pick], loops])
    d2 = np.concatenate([g.b, g.a[pick], loops])
    g2 = oracle.simple_graph(n, s2, d2)
    assert g2.m_hat == g.m_hat
    assert g2.self_loops == 50
    assert g2.duplicates == 300
    assert oracle.count(oracle.oriented_csr(g2)) == T


def test_order_invariance():
    """Sec. III-A: any total order counts each triangle exactly once."""
    n, s, d = _some_graph(5)
    g = oracle.simple_graph(n, s, d)
    T = oracle.count(oracle.oriented_csr(g))
    assert oracle.count(oracle.oriented_csr(g, rank=np.arange(n))) == T
    rng = np.random.default_rng(2)
    for _ in range(3):
        assert oracle.count(oracle.oriented_csr(g, rank=rng.permutation(n))) == T


def test_degree_order_orientation():
    """Each oriented edge (v, u) satisfies d_v < d_u or (d_v = d_u and v < u), and lists are sorted."""
    n, s, d = _some_graph(6)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    deg = csr.deg.astype(np.int64)
    for v in range(n):
        row = csr.cols[csr.off[v]:csr.off[v + 1]]
        assert np.all(np.diff(row) > 0)
        for u in row:
            assert deg[v] < deg[u] or (deg[v] == deg[u] and v < u)
    A = BF.adjacency(n, s, d)
    assert np.array_equal(deg, A.sum(1))
    assert csr.m_hat == int(A.sum()) // 2


def test_theorem1_per_edge_attribution():
    """Theorem 1: the triangle x1 < x2 < x3 (degree order) is found once, on edge (x1, x2)."""
    n, s, d = _some_graph(7)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    T, per_edge, _ = oracle.count(csr, per_edge=True)
    deg = csr.deg

    def key(x):
        return (int(deg[x]), x)

    expect = {}
    for tri in BF.triangle_list(n, s, d):
        x1, x2, _ = sorted(tri, key=key)
        expect[(x1, x2)] = expect.get((x1, x2), 0) + 1
    got = {}
    for v in range(n):
        for i in range(csr.off[v], csr.off[v + 1]):
            if per_edge[i]:
                got[(v, int(csr.cols[i]))] = int(per_edge[i])
    assert got == expect
    assert T == sum(expect.values())


def test_per_vertex_matches_definition():
    n, s, d = _some_graph(8)
    _, _, tv = oracle.count(oracle.oriented_csr(oracle.simple_graph(n, s, d)), per_vertex=True)
    assert np.array_equal(tv.astype(np.int64), BF.per_vertex_by_definition(n, s, d))


def test_threads_give_same_count():
    n, s, d = _some_graph(9)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    assert oracle.count(csr, threads=4) == oracle.count(csr, threads=1)


# --------------------------------------------------------------------------- input policy

def test_input_policy_errors():
    with pytest.raises(oracle.OracleError) as e:
        oracle.simple_graph(5, [0, 1, 5], [1, 2, 0])
    assert e.value.code == oracle.ERR_VERTEX_RANGE
    with pytest.raises(oracle.OracleError) as e:
        oracle.simple_graph(5, [0, -1], [1, 2])
    assert e.value.code == oracle.ERR_VERTEX_RANGE
    with pytest.raises(oracle.OracleError) as e:
        oracle.simple_graph(5, [0, 1, 1], [1, 1, 2], strict=True)
    assert e.value.code == oracle.ERR_INVALID_ARG
    with pytest.raises(oracle.OracleError) as e:
        oracle.simple_graph(5, [0, 1], [1, 0], strict=True)
    assert e.value.code == oracle.ERR_INVALID_ARG
    g = oracle.simple_graph(5, [0, 1, 1, 2, 3], [1, 0, 1, 3, 2])
    assert (g.m_hat, g.self_loops, g.duplicates) == (2, 1, 2)
    assert list(g.a) == [0, 2] and list(g.b) == [1, 3]


def test_empty_inputs():
    assert oracle_T(0, [], []) == 0
    assert oracle_T(10, [], []) == 0
    assert oracle_T(3, [1, 1], [1, 1]) == 0


# --------------------------------------------------------------------------- statistics

def test_er_config0_expected_count():
    """G(n,m) with n=1e4, m=1e5: E[T] = C(n,3) p^3, p = m / C(n,2) (about 1333.6)."""
    from graphgen import workloads as W
    s, d = W.ER_10K.edges()
    n, m = W.ER_10K.n, W.ER_10K.m
    g = oracle.simple_graph(n, s, d)
    assert g.m_hat == m and g.self_loops == 0 and g.duplicates == 0
    T = oracle.count(oracle.oriented_csr(g))
    p = m / math.comb(n, 2)
    mean = math.comb(n, 3) * p ** 3
    # variance of a triangle count in G(n,p): the triangle term plus pairs sharing an edge
    var = mean * (1 - p ** 3) + math.comb(n, 4) * 6 * p ** 5 * (1 - p)
    assert abs(T - mean) < 6 * math.sqrt(var)


# --------------------------------------------------------------------------- partitioned count

def _random_cuts(rng, n, P):
    inner = np.sort(rng.integers(0, n + 1, P - 1))
    return np.array([0, *inner, n], np.int64)


@pytest.mark.parametrize("seed", [10, 11, 12])
def test_partition_table_by_brute_force(seed):
    """Sec. IV-A / IV-C: the triangle x1 < x2 < x3 (degree order) is found once, on the
    oriented edge (x1, x2): by the processor holding x2, in the list N_x1 sent by the
    processor holding x1.  Degrees and parts come from the adjacency matrix here."""
    n, s, d = _some_graph(seed)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    deg = BF.adjacency(n, s, d).sum(1)
    tris = BF.triangle_list(n, s, d)
    rng = np.random.default_rng(seed)
    for P in (1, 2, 3, 5, 8, 40):
        cuts = _random_cuts(rng, n, P)
        part = np.searchsorted(cuts, np.arange(n), side="right") - 1
        expect = np.zeros((P, P), np.int64)
        for tri in tris:
            x1, x2, _ = sorted(tri, key=lambda x: (int(deg[x]), x))
            expect[part[x1], part[x2]] += 1
        got = oracle.count_parts(csr, cuts).astype(np.int64)
        assert np.array_equal(got, expect), (P, cuts)


def test_partition_table_sums_to_T_and_empty_parts():
    import graphgen
    n = 3000
    s, d = graphgen.chung_lu(n, 2.05, 20.0, 600.0, 40_000, 5)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    T = oracle.count(csr)
    assert oracle.count_parts(csr, [0, n]).tolist() == [[T]]
    # empty sets of vertices anywhere, including first and last
    for cuts in ([0, 0, 100, 100, 2999, n, n], [0, 1, 2, 3, n], [0, n, n]):
        tab = oracle.count_parts(csr, cuts)
        assert int(tab.sum()) == T
        sizes = np.diff(cuts)
        assert np.all(tab[sizes == 0, :] == 0) and np.all(tab[:, sizes == 0] == 0)


def test_partition_bad_cuts():
    n, s, d = _some_graph(13)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    for cuts in ([1, n], [0, n - 1], [0, 300, 200, n]):
        with pytest.raises(oracle.OracleError):
            oracle.count_parts(csr, cuts)


# ---------------------------------------------------------------- Sec. IV-B balanced cuts

def _prefix(f):
    F = [0]
    for x in f:
        F.append(F[-1] + int(x))
    return F


@pytest.mark.parametrize("seed", range(12))
def test_balanced_cuts_balance_and_minimality(seed):
    """Every part's cost is below total/P + max f (no cut could move right and keep the parts
    under their share), and no cut can move left: F(c_k - 1) < k/P of the total <= F(c_k)."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    f = rng.integers(0, 50, n).astype(np.uint64)
    f[rng.random(n) < 0.3] = 0
    for P in (1, 2, 3, 7, 16, n, n + 5):
        cuts = oracle.balanced_cuts(f, P).tolist()
        F = _prefix(f)
        tot, fmax = F[-1], int(f.max())
        assert cuts[0] == 0 and cuts[-1] == n and len(cuts) == P + 1
        assert all(a <= b for a, b in zip(cuts, cuts[1:]))
        for k in range(P):
            assert (F[cuts[k + 1]] - F[cuts[k]]) * P <= tot + fmax * P
        for k in range(1, P):
            c = cuts[k]
            assert F[c] * P >= k * tot
            assert c == 0 or F[c - 1] * P < k * tot


def test_balanced_cuts_closed_forms():
    # equal costs, n = a P: parts of exactly a vertices
    for a, P in ((5, 4), (1, 9), (13, 3)):
        assert oracle.balanced_cuts(np.ones(a * P, np.uint64), P).tolist() == list(range(0, a * P + 1, a))
    # one vertex h carries all the cost: every inner cut sits right after it
    n, h = 40, 17
    f = np.zeros(n, np.uint64)
    f[h] = 1000
    assert oracle.balanced_cuts(f, 5).tolist() == [0] + [h + 1] * 4 + [n]
    # no cost at all: the last part takes every vertex
    assert oracle.balanced_cuts(np.zeros(6, np.uint64), 3).tolist() == [0, 0, 0, 6]
    # totals beyond 64 bits once multiplied by P
    big = np.full(4, 2 ** 62, np.uint64)
    assert oracle.balanced_cuts(big, 4).tolist() == [0, 1, 2, 3, 4]
    with pytest.raises(oracle.OracleError):
        oracle.balanced_cuts(np.ones(3, np.uint64), 0)


def test_partition_table_closed_form_on_complete_graph():
    """K_n: all degrees tie, so the order is by id and triangle {x < y < z} is counted by the part
    of its middle vertex y for the part of x.  Entry (i, j) is the number of (x, y, z) with
    x < y < z, x in V_i and y in V_j: the sum over y in V_j of |{x in V_i : x < y}| (n - 1 - y)."""
    from graphgen import families as F
    n, s, d = F.complete(40)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    for cuts in ([0, 40], [0, 7, 7, 20, 33, 40], list(range(0, 41, 5)), [0, 1, 39, 40]):
        P = len(cuts) - 1
        want = np.zeros((P, P), np.int64)
        for i in range(P):
            for j in range(P):
                for y in range(cuts[j], cuts[j + 1]):
                    below = max(0, min(cuts[i + 1], y) - cuts[i])
                    want[i, j] += below * (n - 1 - y)
        got = oracle.count_parts(csr, cuts).astype(np.int64)
        assert np.array_equal(got, want), cuts
        assert int(want.sum()) == n * (n - 1) * (n - 2) // 6
