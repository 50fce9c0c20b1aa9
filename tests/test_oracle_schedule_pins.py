"""Pins of the oracle's cost functions and chunk table.

Cost functions (Sec. IV-B, IV-F, V-A) are checked against their set-builder
definitions evaluated with Python sets; the chunk table (Eq. 1 and Eq. 2 of
Sec. V-B) against worked examples derived by hand and against the properties
the paper states.  The library's own task decomposition is not the oracle's:
its checks are in test_schedule_model.py.
"""
import numpy as np
import pytest

import oracle


def _csr(seed=3, n=300):
    import graphgen
    s, d = graphgen.chung_lu(n, 2.2, 12.0, 90.0, n * 6, seed)
    return n, s, d, oracle.oriented_csr(oracle.simple_graph(n, s, d))


def _sets(csr):
    n = csr.n
    Nplus = [set(csr.cols[csr.off[v]:csr.off[v + 1]].tolist()) for v in range(n)]
    Nfull = [set() for _ in range(n)]
    for v in range(n):
        for u in Nplus[v]:
            Nfull[v].add(u)
            Nfull[u].add(v)
    return Nplus, Nfull


def test_vertex_cost_definitions():
    n, s, d, csr = _csr()
    Nplus, Nfull = _sets(csr)
    dh = [len(x) for x in Nplus]
    f1 = oracle.vertex_cost(csr, oracle.COST_ONE)
    fd = oracle.vertex_cost(csr, oracle.COST_DEGREE)
    fp = oracle.vertex_cost(csr, oracle.COST_PATRIC)
    fn = oracle.vertex_cost(csr, oracle.COST_NEW)
    for v in range(n):
        assert f1[v] == 1
        assert fd[v] == len(Nfull[v])
        assert fp[v] == sum(dh[v] + dh[u] for u in Nplus[v])
        assert fn[v] == sum(dh[v] + dh[u] for u in Nfull[v] - Nplus[v])
    # both estimates charge every oriented edge (v, u) exactly dh_v + dh_u, to v or to u
    assert int(fp.sum()) == int(fn.sum())
    assert int(fd.sum()) == 2 * csr.m_hat


def test_schedule_unit_costs_worked_example():
    """100 tasks of cost 1, W = 4, floor 1.  C = 100, H = 50.
    Eq. 1: 50 = 4*12 + 2 -> static chunks of 13, 13, 12, 12 tasks.
    Eq. 2 from c = 50: floor(50/4)=12, floor(38/4)=9, floor(29/4)=7, floor(22/4)=5,
    floor(17/4)=4, floor(13/4)=3, floor(10/4)=2, floor(8/4)=2, floor(6/4)=1,
    floor(5/4)=1, floor(4/4)=1, then the floor of 1 for the last three."""
    cb, tb = oracle.schedule(np.ones(100, np.uint64), 4, 1)
    sizes = np.diff(tb).tolist()
    assert sizes == [13, 13, 12, 12, 12, 9, 7, 5, 4, 3, 2, 2, 1, 1, 1, 1, 1, 1]
    assert np.array_equal(cb, tb.astype(np.uint64))


def test_schedule_single_worker():
    """W = 1: Eq. 1 gives one task of half the cost, Eq. 2 gives the whole rest at once."""
    cost = np.arange(1, 41, dtype=np.uint64)
    C = int(cost.sum())
    cb, tb = oracle.schedule(cost, 1, 1)
    assert cb.tolist() == [0, C // 2, C]
    prefix = np.concatenate([[0], np.cumsum(cost)])
    assert tb[1] == int(np.searchsorted(prefix[:-1], C // 2, side="left"))
    assert tb[0] == 0 and tb[-1] == 40


def test_schedule_min_chunk_floor_and_edge_cases():
    cb, tb = oracle.schedule(np.ones(10, np.uint64), 3, 100)
    # H = 5 split 2,2,1; the remaining 5 < floor -> one chunk
    assert np.diff(tb).tolist() == [2, 2, 1, 5]
    cb, tb = oracle.schedule(np.zeros(0, np.uint64), 8, 16)
    assert tb.tolist() == [0] * 9
    # all-zero costs: everything lands in the first chunk
    cb, tb = oracle.schedule(np.zeros(5, np.uint64), 2, 1)
    assert tb[0] == 0 and tb[1] == 5 and tb[-1] == 5


@pytest.mark.parametrize("W,minc", [(7, 1), (64, 8), (152, 50)])
def test_schedule_properties(W, minc):
    # uneven costs: the merge cost d^_v + d^_u of every oriented edge (Sec. III-A) of a skewed graph
    n, s, d, csr = _csr(5, 2000)
    dh = np.diff(csr.off)
    rows = np.repeat(np.arange(n), dh)
    cost = (dh[rows] + dh[csr.cols]).astype(np.uint64)
    cb, tb = oracle.schedule(cost, W, minc)
    C = int(cost.sum())
    T = len(cost)
    assert tb[0] == 0 and tb[-1] == T and np.all(np.diff(tb) >= 0)
    assert cb[0] == 0 and int(cb[-1]) == C and np.all(np.diff(cb.astype(np.int64)) >= 0)
    assert int(cb[W]) == C // 2
    prefix = np.concatenate([[0], np.cumsum(cost.astype(np.int64))])
    cmax = int(cost.max())
    for k in range(len(cb) - 1):
        got = int(prefix[tb[k + 1]] - prefix[tb[k]])
        want = int(cb[k + 1]) - int(cb[k])
        assert abs(got - want) <= cmax  # snapping to task boundaries moves each end by < one task
    static = np.diff(cb[:W + 1].astype(np.int64))
    assert static.max() - static.min() <= 1  # Eq. 1: equal initial tasks
    dyn = np.diff(cb[W:].astype(np.int64))
    assert np.all(dyn[:-1] >= minc)
    assert np.all(np.diff(dyn[:-1]) <= 0)  # Eq. 2: task sizes never grow
