"""CPU oracle for exact triangle counting -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs it, and it shares no code with
that path.

The arithmetic lives in ``tc_oracle.c`` (plain sequential C following Fig. 1
of the paper and its definitions; see that file's header).  This module only
compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tc_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libtc_oracle.so")
_lib = None
_lock = threading.Lock()

OK, ERR_INVALID_ARG, ERR_VERTEX_RANGE, ERR_OOM = 0, 1, 2, 3
COST_ONE, COST_DEGREE, COST_PATRIC, COST_NEW = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"oracle error {code}: {msg}")
        self.code = code


class _Stats(ctypes.Structure):
    _fields_ = [("m_in", ctypes.c_int64), ("self_loops", ctypes.c_int64),
                ("duplicates", ctypes.c_int64), ("m_hat", ctypes.c_int64),
                ("bad_index", ctypes.c_int64)]


def build(force: bool = False) -> str:
    """Compile ``libtc_oracle.so`` next to its source (gcc -O2, OpenMP for the optional threads)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            P = ctypes.c_void_p
            i32, i64, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
            L.or_simple_graph.argtypes = [i32, i64, P, P, ctypes.c_int, P, P, ctypes.POINTER(_Stats)]
            L.or_simple_graph.restype = ctypes.c_int
            L.or_oriented_csr.argtypes = [i32, i64, P, P, P, P, P, P]
            L.or_oriented_csr.restype = ctypes.c_int
            L.or_count.argtypes = [i32, P, P, P, P, ctypes.c_int]
            L.or_count.restype = u64
            L.or_count_parts.argtypes = [i32, P, P, i32, P, P]
            L.or_count_parts.restype = ctypes.c_int
            L.or_balanced_cuts.argtypes = [i32, P, i32, P]
            L.or_balanced_cuts.restype = ctypes.c_int
            L.or_vertex_cost.argtypes = [ctypes.c_int, i32, P, P, P, P]
            L.or_vertex_cost.restype = ctypes.c_int
            L.or_schedule.argtypes = [i64, P, i64, u64, P, P, i64]
            L.or_schedule.restype = i64
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class SimpleGraph:
    n: int
    a: np.ndarray   # int32, a < b, sorted by (a, b)
    b: np.ndarray
    self_loops: int
    duplicates: int

    @property
    def m_hat(self) -> int:
        return len(self.a)


@dataclass
class OrientedCSR:
    n: int
    deg: np.ndarray   # int32 [n]      d_v
    off: np.ndarray   # int64 [n+1]
    cols: np.ndarray  # int32 [m_hat]  N_v = cols[off[v]:off[v+1]], ascending

    @property
    def m_hat(self) -> int:
        return int(self.off[-1])

    @property
    def dhat(self) -> np.ndarray:
        return np.diff(self.off)


def simple_graph(n, src, dst, strict=False) -> SimpleGraph:
    """Sec. II input model: drop self-loops and merge repeated/reversed pairs (or reject if strict)."""
    L = _load()
    src = np.ascontiguousarray(src, dtype=np.int32)
    dst = np.ascontiguousarray(dst, dtype=np.int32)
    m = len(src)
    ea = np.empty(max(m, 1), np.int32)
    eb = np.empty(max(m, 1), np.int32)
    st = _Stats()
    rc = L.or_simple_graph(n, m, _p(src), _p(dst), int(bool(strict)), _p(ea), _p(eb), ctypes.byref(st))
    if rc != OK:
        raise OracleError(rc, f"bad_index={st.bad_index} self_loops={st.self_loops} duplicates={st.duplicates}")
    k = st.m_hat
    return SimpleGraph(n, ea[:k].copy(), eb[:k].copy(), st.self_loops, st.duplicates)


def oriented_csr(g: SimpleGraph, rank=None) -> OrientedCSR:
    """Fig. 1, first two loops: orient by the degree order (or by `rank`) and sort each N_v."""
    L = _load()
    n, mh = g.n, g.m_hat
    deg = np.empty(max(n, 1), np.int32)
    off = np.empty(n + 1, np.int64)
    cols = np.empty(max(mh, 1), np.int32)
    rk = None if rank is None else np.ascontiguousarray(rank, dtype=np.int64)
    rc = L.or_oriented_csr(n, mh, _p(g.a), _p(g.b), _p(rk), _p(deg), _p(off), _p(cols))
    if rc != OK:
        raise OracleError(rc)
    return OrientedCSR(n, deg[:n], off, cols[:mh])


def count(csr: OrientedCSR, per_edge=False, per_vertex=False, threads=1):
    """Fig. 1, last loop.  Returns T, or (T, per_edge uint32[m_hat] | None, t_v uint64[n] | None)."""
    L = _load()
    pe = np.zeros(max(csr.m_hat, 1), np.uint32) if per_edge else None
    tv = np.zeros(max(csr.n, 1), np.uint64) if per_vertex else None
    T = int(L.or_count(csr.n, _p(csr.off), _p(csr.cols), _p(pe), _p(tv), int(threads)))
    if not per_edge and not per_vertex:
        return T
    return T, (pe[:csr.m_hat] if per_edge else None), (tv[:csr.n] if per_vertex else None)


def count_parts(csr: OrientedCSR, cuts) -> np.ndarray:
    """Sec. IV-A / IV-C: the P x P table of SurrogateCount sums over the non-overlapping
    partition with vertex sets [cuts[j], cuts[j+1]): entry (i, j) is what processor j counts
    for the lists N_v, v in V_i, that it receives.  The table sums to T."""
    L = _load()
    cuts = np.ascontiguousarray(cuts, dtype=np.int32)
    P = len(cuts) - 1
    out = np.zeros(max(P, 1) * max(P, 1), np.uint64)
    rc = L.or_count_parts(csr.n, _p(csr.off), _p(csr.cols), P, _p(cuts), _p(out))
    if rc != OK:
        raise OracleError(rc, "bad cuts")
    return out[:P * P].reshape(P, P)


def balanced_cuts(f, P: int) -> np.ndarray:
    """Sec. IV-B: cuts (P + 1 int32) of V into P sets of consecutive vertices of about equal cost:
    cut k is the first q whose cost prefix f(0) + ... + f(q-1) reaches k/P of the total."""
    L = _load()
    f = np.ascontiguousarray(f, dtype=np.uint64)
    cuts = np.zeros(int(P) + 1, np.int32)
    rc = L.or_balanced_cuts(len(f), _p(f), int(P), _p(cuts))
    if rc != OK:
        raise OracleError(rc, "bad part count")
    return cuts


def count_edges(n, src, dst, strict=False, threads=1) -> int:
    """End to end: simple graph -> oriented lists -> T."""
    return count(oriented_csr(simple_graph(n, src, dst, strict)), threads=threads)


def vertex_cost(csr: OrientedCSR, fn: int) -> np.ndarray:
    """Per-vertex f(v) for fn in COST_ONE, COST_DEGREE, COST_PATRIC, COST_NEW."""
    L = _load()
    f = np.zeros(max(csr.n, 1), np.uint64)
    rc = L.or_vertex_cost(int(fn), csr.n, _p(csr.deg), _p(csr.off), _p(csr.cols), _p(f))
    if rc != OK:
        raise OracleError(rc)
    return f[:csr.n]


def schedule(cost, workers: int, min_chunk: int):
    """Chunk table (Eq. 1 static half + Eq. 2 guided rest): (cost bounds uint64[K+1], task bounds int64[K+1])."""
    L = _load()
    cost = np.ascontiguousarray(cost, np.uint64)
    T = len(cost)
    total = int(cost.sum(dtype=np.uint64)) if T else 0
    # static W+1 boundaries plus at most (remaining / min_chunk) + W*64 guided ones
    cap = workers + 2 + total // max(min_chunk, 1) + 64 * workers + 64
    cap = int(min(cap, 1 << 26))
    cb = np.empty(cap, np.uint64)
    tb = np.empty(cap, np.int64)
    k = L.or_schedule(T, _p(cost), int(workers), int(min_chunk), _p(cb), _p(tb), cap)
    if k < 0:
        raise OracleError(ERR_INVALID_ARG, "schedule capacity")
    return cb[:k + 1].copy(), tb[:k + 1].copy()
