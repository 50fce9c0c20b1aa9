"""Checks of tests/schedule_model.py, the library's own decomposition restated for the tests.

The decomposition is this design's, not the paper's, so these are not pins of the oracle.
They fix the definitions the GPU's task array and chunk table are compared with: every
oriented edge of Fig. 1 becomes one task (or is dropped when it can count nothing), the
tasks preserve the count (Theorem 1), the order and classes are as stated, and hand-worked
examples fix the task costs.
"""
import numpy as np
import pytest

import oracle
from graphgen import families as F

from tests import schedule_model as M


def _csr(seed=3, n=300):
    import graphgen
    s, d = graphgen.chung_lu(n, 2.2, 12.0, 90.0, n * 6, seed)
    return n, s, d, oracle.oriented_csr(oracle.simple_graph(n, s, d))


def _nplus(csr):
    return [set(csr.cols[csr.off[v]:csr.off[v + 1]].tolist()) for v in range(csr.n)]


def test_tasks_cover_each_oriented_edge_once_and_preserve_the_count():
    n, s, d, csr = _csr(4)
    Nplus = _nplus(csr)
    dh = np.diff(csr.off)
    owner, partner, pos = M.tasks(csr, with_pos=True)
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
    owner, partner = M.tasks(csr)
    assert list(zip(owner.tolist(), partner.tolist())) == [(1, 2), (1, 5), (2, 3), (3, 4), (4, 5)]
    # EDGE model with piece=2, c_task=4, c_owner=32:
    #   (1,2): pieces(3)=2 -> 2*(2+4)=12;  (1,5): 2*(1+4)=10, last of owner 1: + 3+32 -> 45
    #   (2,3): 1*(2+4)=6 + 2+32 -> 40;  (3,4): 6+34 -> 40;  (4,5): 1*(1+4)=5 + 34 -> 39
    c = M.task_costs(csr, owner, partner, M.MODEL_EDGE, piece=2, c_task=4, c_owner=32)
    assert list(c) == [12, 45, 40, 40, 39]
    # MERGE model: dh_o + dh_p
    c = M.task_costs(csr, owner, partner, M.MODEL_MERGE)
    assert list(c) == [5, 4, 4, 4, 3]
    # VERTEX model, f = d_v: only the last task of each owner carries f(owner) = 3
    c = M.task_costs(csr, owner, partner, M.MODEL_VERTEX, fn=oracle.COST_DEGREE)
    assert list(c) == [0, 3, 3, 3, 3]


def test_task_costs_with_classes_worked_example():
    """W_6 again, with small_max = 2: owner 1 (list of 3) is big, owners 2, 3, 4 are small.
    Order: small (2,3) (3,4) (4,5), then big (1,2) (1,5).
    EDGE, piece = 2, c_task = 4, c_owner = 32 (small owners take one piece):
      (2,3): 1*(2+4) + 2+32 = 40; (3,4): 40; (4,5): 1*(1+4) + 34 = 39;
      (1,2): 2*(2+4) = 12; (1,5): 2*(1+4) + 3+32 = 45."""
    n, s, d = F.wheel(6)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    o, p, ns = M.tasks(csr, small_max=2, with_split=True)
    assert ns == 3
    assert list(zip(o.tolist(), p.tolist())) == [(2, 3), (3, 4), (4, 5), (1, 2), (1, 5)]
    c = M.task_costs(csr, o, p, M.MODEL_EDGE, piece=2, c_task=4, c_owner=32, small_max=2)
    assert list(c) == [40, 40, 39, 12, 45]


def test_vertex_model_chunks_never_split_an_owner():
    n, s, d, csr = _csr(6, 1500)
    owner, partner = M.tasks(csr)
    for fn in (oracle.COST_ONE, oracle.COST_DEGREE, oracle.COST_PATRIC):
        cost = M.task_costs(csr, owner, partner, M.MODEL_VERTEX, fn=fn)
        cb, tb = oracle.schedule(cost, 16, 1)
        for t in tb[1:-1]:
            if 0 < t < len(owner):
                assert owner[t] != owner[t - 1]


def test_task_classes_split_by_owner_list_length():
    n, s, d, csr = _csr(8, 800)
    dh = np.diff(csr.off)
    o_all, p_all = M.tasks(csr)
    for k in (0, 3, 8, 20, 10**9):
        o, p, ns = M.tasks(csr, small_max=k, with_split=True)
        assert set(zip(o.tolist(), p.tolist())) == set(zip(o_all.tolist(), p_all.tolist()))
        assert np.all(dh[o[:ns]] <= k) and np.all(dh[o[ns:]] > k)
        _, _, pos = M.tasks(csr, small_max=k, with_pos=True)
        for lo, hi in ((0, ns), (ns, len(o))):
            key = o[lo:hi].astype(np.int64) * (csr.m_hat + 1) + pos[lo:hi]
            assert np.all(np.diff(key) > 0)


def test_partition_members_worked_example():
    """Costs [3, 0, 4, 1, 2, 0] (C = 10, exclusive prefixes 0 3 3 7 8 10) in 3 parts
    [0, 3) [3, 6) [6, 10]: tasks 0 | 1 2 | 3 4 5 (the zero-cost task at C goes last)."""
    part = M.partition_members(np.array([3, 0, 4, 1, 2, 0], np.uint64), 3)
    assert part.tolist() == [0, 1, 1, 2, 2, 2]
    # more parts than cost units: empty parts, every task in exactly one part
    part = M.partition_members(np.array([1, 1], np.uint64), 5)
    # C = 2, bounds 0 0 0 1 1 2: parts 0, 1 and 3 are empty, [0, 1) is part 2, [1, 2) part 4
    assert part.tolist() == [2, 4]
    assert M.partition_members(np.zeros(0, np.uint64), 4).tolist() == []


@pytest.mark.parametrize("nparts", [1, 2, 3, 7, 64])
def test_partition_members_cover_tasks_in_order(nparts):
    n, s, d, csr = _csr(9, 1200)
    owner, partner = M.tasks(csr)
    cost = M.task_costs(csr, owner, partner, M.MODEL_EDGE, piece=16)
    part = M.partition_members(cost, nparts)
    assert np.all(np.diff(part) >= 0) and part.min() >= 0 and part.max() < nparts
    C = int(cost.sum())
    for k in range(nparts):
        got = int(cost[part == k].sum())
        assert abs(got - C / nparts) <= int(cost.max()) + 1
