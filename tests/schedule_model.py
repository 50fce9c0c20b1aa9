"""This library's own work decomposition and task costs, restated in numpy for the tests.

NOT THE ORACLE.  The paper defines neither the decomposition nor the EDGE cost below: they are
this design's choices.  The module exists so that the tests can check the GPU's task array,
chunk table and task partition against an independent statement of the same definitions.  It
takes from the oracle only what the paper does define: the oriented lists (Fig. 1), the
per-vertex cost functions (Sec. IV-B, IV-F, V-A) and, through the tests, the Eq. 1 / Eq. 2
chunk table (Sec. V-B) over a cost sequence.

The decomposition.  Each oriented edge (v, u) of Fig. 1 is one task, counted as
|N_v ∩ N_u| (Theorem 1: every triangle once).  Its owner is the endpoint with the longer
list (v on a tie) and its partner the other endpoint.  A task whose partner list is empty
counts nothing and is dropped.  A task is "small" when its owner's list has at most
small_max entries, else "big".  Tasks are ordered by (class, owner, position of the oriented
edge in the lists).

Task costs.
  EDGE   this design's hash work: the owner's list is staged in pieces of at most `piece`
         entries (one piece for a small owner) and every partner list is streamed once per
         piece, so a task costs pieces(owner) * (dh_partner + c_task); the owner's last task
         also carries its staging, dh_owner + c_owner.
  MERGE  the paper's merge cost of an oriented edge, dh_v + dh_u (Sec. III-A).
  VERTEX a per-vertex cost f(owner) of the paper, put on the owner's last task so that a chunk
         never splits an owner (the atomic task <v,1> of Sec. V-A).
"""
from __future__ import annotations

import numpy as np

import oracle

MODEL_EDGE = 0
MODEL_MERGE = 1
MODEL_VERTEX = 2


def tasks(csr, small_max: int = 1 << 40, with_split: bool = False, with_pos: bool = False):
    """(owner int32[T], partner int32[T]) in task order; with_split adds the number of small
    tasks, with_pos the position of each task's oriented edge in csr.cols."""
    off = np.asarray(csr.off, np.int64)
    cols = np.asarray(csr.cols, np.int64)
    dh = np.diff(off)
    row = np.repeat(np.arange(csr.n, dtype=np.int64), dh)
    pos = np.arange(len(cols), dtype=np.int64)
    row_owns = dh[row] >= dh[cols]
    owner = np.where(row_owns, row, cols)
    partner = np.where(row_owns, cols, row)
    keep = dh[partner] > 0
    owner, partner, pos = owner[keep], partner[keep], pos[keep]
    big = (dh[owner] > small_max).astype(np.int64)
    order = np.lexsort((pos, owner, big))
    owner, partner, pos = owner[order], partner[order], pos[order]
    out = [owner.astype(np.int32), partner.astype(np.int32)]
    if with_split:
        out.append(int((big == 0).sum()))
    if with_pos:
        out.append(pos)
    return tuple(out)


def task_costs(csr, owner, partner, model=MODEL_EDGE, fn=oracle.COST_DEGREE, piece=1024, c_task=4, c_owner=32,
               small_max: int = 0) -> np.ndarray:
    """uint64 cost of every task under `model` (see the module text)."""
    off = np.asarray(csr.off, np.int64)
    dh = np.diff(off)
    o = np.asarray(owner, np.int64)
    p = np.asarray(partner, np.int64)
    T = len(o)
    dho, dhp = dh[o].astype(np.uint64), dh[p].astype(np.uint64)
    last = np.ones(T, bool)
    if T > 1:
        last[:-1] = o[1:] != o[:-1]
    if model == MODEL_EDGE:
        if piece < 1:
            raise ValueError("piece must be positive")
        pieces = np.where(dho <= np.uint64(small_max), np.uint64(1),
                          (dho + np.uint64(piece - 1)) // np.uint64(piece))
        cost = pieces * (dhp + np.uint64(c_task))
        cost = cost + np.where(last, dho + np.uint64(c_owner), np.uint64(0))
    elif model == MODEL_MERGE:
        cost = dho + dhp
    elif model == MODEL_VERTEX:
        f = oracle.vertex_cost(csr, fn)
        cost = np.where(last, f[o] if T else np.zeros(0, np.uint64), np.uint64(0))
    else:
        raise ValueError("unknown cost model")
    return np.asarray(cost, np.uint64)


def partition_members(cost, nparts: int):
    """Part index of every task of one class when the class's cost is cut into nparts ranges
    [C p / P, C (p + 1) / P): a task belongs to the part whose range holds its exclusive cost
    prefix; prefixes at C (zero-cost tasks at the end) belong to the last part."""
    cost = np.asarray(cost, np.uint64)
    excl = np.concatenate([np.zeros(1, np.uint64), np.cumsum(cost, dtype=np.uint64)])[:-1]
    C = int(cost.sum(dtype=np.uint64)) if len(cost) else 0
    bounds = np.array([C * k // nparts for k in range(nparts + 1)], np.uint64)
    part = np.searchsorted(bounds, excl, side="right").astype(np.int64) - 1
    return np.minimum(part, nparts - 1)
