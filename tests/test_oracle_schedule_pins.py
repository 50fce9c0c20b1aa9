"""Pins of the oracle's cost functions, task decomposition and chunk table.

Cost functions (Sec. IV-B, IV-F, V-A) are checked against their set-builder
definitions evaluated with Python sets; the task decomposition against the
count it must preserve; the chunk table (Eq. 1 and Eq. 2 of Sec. V-B) against
worked examples derived by hand and against the properties the paper states.
"""
import numpy as np
import pytest

import oracle
from graphgen import families as F


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


def test_tasks_cover_each_oriented_edge_once_and_preserve_the_count():
    n, s, d, csr = _csr(4)
    Nplus, _ = _sets(csr)
    dh = np.diff(csr.off)
    owner, partner, pos = oracle.tasks(csr, with_pos=True)
    keys = owner.astype(np.int64) * (csr.m_hat + 1) + pos
    assert np.all(np.diff(keys) > 0)  # sorted by (owner, position of the oriented edge), no repeats
    rows = np.searchsorted(csr.off, pos, side="right") - 1
    for o_, p_, i_, r_ in zip(owner.tolist(), partner.tolist(), pos.tolist(), rows.tolist()):
        assert {o_, p_} == {r_, int(csr.cols[i_])}  # the task is the oriented edge at position i_
    seen = set()
    for o, p in zip(owner.tolist(), partner.tolist()):
        assert dh[o] >= dh[p] >= 1
        edge = (o, p) if p in Nplus[o] else (p, o)
        assert edge[1] in Nplus[edge[0]]
        # ties go to the lower endpoint of the oriented edge
        if dh[o] == dh[p]:
            assert edge[0] == o
        seen.add(edge)
    expect = {(v, u) for v in range(n) for u in Nplus[v] if min(dh[v], dh[u]) > 0}
    assert seen == expect
    T = oracle.count(csr)
    assert sum(len(Nplus[o] & Nplus[p]) for o, p in zip(owner.tolist(), partner.tolist())) == T


def test_task_costs_worked_example():
    """Wheel W_6: hub 0, rim 1-2-3-4-5-1.  Degrees: hub 5, rim 3.
    Order: rim vertices by id, then the hub.  Oriented lists:
      N_1 = {2, 5, 0}, N_2 = {3, 0}, N_3 = {4, 0}, N_4 = {5, 0}, N_5 = {0}, N_0 = {}.
    dh = [0, 3, 2, 2, 2, 1].  Oriented edges and their tasks (owner has the longer list):
      (1,2)->(1,2) (1,5)->(1,5) (1,0)->partner 0 has an empty list: dropped
      (2,3)->(2,3) (2,0) dropped  (3,4)->(3,4) (3,0) dropped  (4,5)->(4,5) (4,0) dropped
      (5,0) dropped.
    Tasks sorted: (1,2) (1,5) (2,3) (3,4) (4,5); each intersection is {0}, so T = 5.
    """
    n, s, d = F.wheel(6)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    assert list(np.diff(csr.off)) == [0, 3, 2, 2, 2, 1]
    owner, partner = oracle.tasks(csr)
    assert list(zip(owner.tolist(), partner.tolist())) == [(1, 2), (1, 5), (2, 3), (3, 4), (4, 5)]
    # EDGE model with piece=2, c_task=4, c_owner=32:
    #   (1,2): pieces(3)=2 -> 2*(2+4)=12;  (1,5): 2*(1+4)=10, last of owner 1: + 3+32 -> 45
    #   (2,3): 1*(2+4)=6 + 2+32 -> 40;  (3,4): 6+34 -> 40;  (4,5): 1*(1+4)=5 + 34 -> 39
    c = oracle.task_costs(csr, owner, partner, oracle.MODEL_EDGE, piece=2, c_task=4, c_owner=32)
    assert list(c) == [12, 45, 40, 40, 39]
    # MERGE model: dh_o + dh_p
    c = oracle.task_costs(csr, owner, partner, oracle.MODEL_MERGE)
    assert list(c) == [5, 4, 4, 4, 3]
    # VERTEX model, f = d_v: only the last task of each owner carries f(owner) = 3
    c = oracle.task_costs(csr, owner, partner, oracle.MODEL_VERTEX, fn=oracle.COST_DEGREE)
    assert list(c) == [0, 3, 3, 3, 3]


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
    n, s, d, csr = _csr(5, 2000)
    owner, partner = oracle.tasks(csr)
    cost = oracle.task_costs(csr, owner, partner, oracle.MODEL_EDGE, piece=16)
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


def test_vertex_model_chunks_never_split_an_owner():
    n, s, d, csr = _csr(6, 1500)
    owner, partner = oracle.tasks(csr)
    for fn in (oracle.COST_ONE, oracle.COST_DEGREE, oracle.COST_PATRIC):
        cost = oracle.task_costs(csr, owner, partner, oracle.MODEL_VERTEX, fn=fn)
        cb, tb = oracle.schedule(cost, 16, 1)
        for t in tb[1:-1]:
            if 0 < t < len(owner):
                assert owner[t] != owner[t - 1]


def test_task_classes_split_by_owner_list_length():
    n, s, d, csr = _csr(8, 800)
    dh = np.diff(csr.off)
    o_all, p_all = oracle.tasks(csr)
    for k in (0, 3, 8, 20, 10**9):
        o, p, ns = oracle.tasks(csr, small_max=k, with_split=True)
        assert set(zip(o.tolist(), p.tolist())) == set(zip(o_all.tolist(), p_all.tolist()))
        assert np.all(dh[o[:ns]] <= k) and np.all(dh[o[ns:]] > k)
        _, _, pos = oracle.tasks(csr, small_max=k, with_pos=True)
        for lo, hi in ((0, ns), (ns, len(o))):
            key = o[lo:hi].astype(np.int64) * (csr.m_hat + 1) + pos[lo:hi]
            assert np.all(np.diff(key) > 0)


def test_task_costs_with_classes_worked_example():
    """W_6 again, with small_max = 2: owner 1 (list of 3) is big, owners 2, 3, 4 are small.
    Order: small (2,3) (3,4) (4,5), then big (1,2) (1,5).
    EDGE, piece = 2, c_task = 4, c_owner = 32 (small owners take one piece):
      (2,3): 1*(2+4) + 2+32 = 40; (3,4): 40; (4,5): 1*(1+4) + 34 = 39;
      (1,2): 2*(2+4) = 12; (1,5): 2*(1+4) + 3+32 = 45."""
    n, s, d = F.wheel(6)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    o, p, ns = oracle.tasks(csr, small_max=2, with_split=True)
    assert ns == 3
    assert list(zip(o.tolist(), p.tolist())) == [(2, 3), (3, 4), (4, 5), (1, 2), (1, 5)]
    c = oracle.task_costs(csr, o, p, oracle.MODEL_EDGE, piece=2, c_task=4, c_owner=32, small_max=2)
    assert list(c) == [40, 40, 39, 12, 45]
