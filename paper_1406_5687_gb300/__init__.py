"""GB300-native exact triangle counting (degree-ordered node-iterator, arXiv 1406.5687).

Thin Python layer over the C ABI of ``include/tc.h``: every computation runs in the
CUDA library ``libtcgb300.so``.  PyTorch supplies device memory and streams.

    import paper_1406_5687_gb300 as tc
    g = tc.Graph.build(src, dst, n)      # numpy int32 (host) or torch int32 CUDA tensors
    T = g.count()
"""
from __future__ import annotations

import ctypes

from . import _lib
from ._lib import (TC_COST_DEGREE, TC_COST_EDGE, TC_COST_MERGE, TC_COST_NEW, TC_COST_ONE, TC_COST_PATRIC,
                   TC_FN_DEGREE, TC_FN_LIST, TC_FN_NEW, TC_FN_ONE, TC_FN_PATRIC, TC_INPUT_SANITIZE, TC_INPUT_STRICT, TcError,
                   default_options)

__all__ = ["Graph", "Batch", "autotune", "Server", "TcError", "default_options", "load", "version", "kernel_launches",
           "count_graphs", "count_surrogate", "surrogate_plan"]


def load():
    """Load the CUDA library (building it in-tree first if needed)."""
    return _lib.load()


def version() -> str:
    return load().tc_version().decode()


def kernel_launches() -> int:
    """Kernels the CUDA library has launched in this process so far."""
    return int(load().tc_kernel_launches())


class _CudaArray:
    """Zero-copy view of library-owned device memory for torch.as_tensor."""

    def __init__(self, ptr: int, n: int, typestr: str):
        self.__cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                         "version": 3, "strides": None}


def _torch():
    import torch
    return torch


def _stream(stream):
    if stream is None:
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _view(ptr, n, typestr):
    torch = _torch()
    if n == 0:
        return torch.empty(0, dtype={"<i4": torch.int32, "<i8": torch.int64}[typestr], device="cuda")
    return torch.as_tensor(_CudaArray(ptr, n, typestr), device="cuda")


def _edge_ptrs(src, dst):
    """(src_ptr, dst_ptr, m, keepalive) for numpy int32 arrays or torch int32 tensors (host or CUDA)."""
    try:
        import torch
        is_t = isinstance(src, torch.Tensor)
    except ImportError:  # pragma: no cover
        is_t = False
    if is_t:
        if src.dtype != torch.int32 or dst.dtype != torch.int32:
            raise TypeError("edge tensors must be int32")
        s, d = src.contiguous(), dst.contiguous()
        return ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(d.data_ptr()), int(s.numel()), (s, d)
    import numpy as np
    s = np.ascontiguousarray(src, dtype=np.int32)
    d = np.ascontiguousarray(dst, dtype=np.int32)
    if s.shape != d.shape:
        raise ValueError("src and dst differ in length")
    return s.ctypes.data_as(ctypes.c_void_p), d.ctypes.data_as(ctypes.c_void_p), int(s.size), (s, d)


class Graph:
    """A graph built on the device: N+ lists of Fig. 1 plus the owner-grouped task array."""

    def __init__(self, handle: ctypes.c_void_p):
        self._h = handle

    # ------------------------------------------------------------------ build / free
    @classmethod
    def build(cls, src, dst, n: int, options: _lib.Options | None = None, stream=None) -> "Graph":
        lib = load()
        sp, dp, m, keep = _edge_ptrs(src, dst)
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        rc = lib.tc_build(sp, dp, m, int(n), opt, _stream(stream), ctypes.byref(h))
        del keep
        _lib.check(rc, "tc_build")
        return cls(h)

    @classmethod
    def build_pairs(cls, edges, n: int, options: _lib.Options | None = None, stream=None) -> "Graph":
        """Build from interleaved pairs: `edges` is an (m, 2) int32 numpy array or torch tensor
        (host or CUDA), edge i being (edges[i, 0], edges[i, 1])."""
        lib = load()
        ep, size, keep = _array_ptr(edges, "int32")
        if size % 2:
            raise ValueError("interleaved pairs need an even number of ids")
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        rc = lib.tc_build_pairs(ep, size // 2, int(n), opt, _stream(stream), ctypes.byref(h))
        del keep
        _lib.check(rc, "tc_build_pairs")
        return cls(h)

    def free(self):
        if self._h:
            load().tc_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # ------------------------------------------------------------------ counts
    def count(self, stream=None) -> int:
        t = ctypes.c_uint64()
        _lib.check(load().tc_count(self._h, _stream(stream), ctypes.byref(t)), "tc_count")
        return int(t.value)

    def count_partition(self, part: int, nparts: int, stream=None) -> int:
        """The count of part `part` of `nparts` cost-balanced parts of the tasks; the parts sum to T."""
        t = ctypes.c_uint64()
        _lib.check(load().tc_count_partition(self._h, int(part), int(nparts), _stream(stream), ctypes.byref(t)),
                   "tc_count_partition")
        return int(t.value)

    def count_async(self, out, stream=None):
        """Enqueue the count; `out` is a CUDA int64 tensor with at least one element."""
        _lib.check(load().tc_count_async(self._h, _stream(stream), ctypes.c_void_p(out.data_ptr())),
                   "tc_count_async")

    def count_static(self, out, stream=None):
        """Enqueue the count without allocating (scratch in the library's fixed device array);
        `out` is a CUDA int64 tensor with at least one element."""
        _lib.check(load().tc_count_static(self._h, _stream(stream), ctypes.c_void_p(out.data_ptr())),
                   "tc_count_static")

    def check(self, stream=None):
        _lib.check(load().tc_graph_check(self._h, _stream(stream)), "tc_graph_check")

    def count_per_vertex(self, stream=None):
        """(T, t_v) with t_v an int64 CUDA tensor of n per-vertex counts (Sec. II)."""
        torch = _torch()
        n = self.info()["n"]
        tv = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        t = ctypes.c_uint64()
        _lib.check(load().tc_count_per_vertex(self._h, _stream(stream), ctypes.c_void_p(tv.data_ptr()),
                                              ctypes.byref(t)), "tc_count_per_vertex")
        return int(t.value), tv[:n]

    def count_per_edge(self, stream=None):
        """(T, c) with c an int32 CUDA tensor: the count of each oriented edge in CSR order."""
        torch = _torch()
        mh = self.info()["m_hat"]
        c = torch.empty(max(mh, 1), dtype=torch.int32, device="cuda")
        t = ctypes.c_uint64()
        _lib.check(load().tc_count_per_edge(self._h, _stream(stream), ctypes.c_void_p(c.data_ptr()),
                                            ctypes.byref(t)), "tc_count_per_edge")
        return int(t.value), c[:mh]

    def clustering(self, t_v, stream=None):
        """Local clustering coefficients (float64 CUDA tensor) from per-vertex counts."""
        torch = _torch()
        n = self.info()["n"]
        cc = torch.empty(max(n, 1), dtype=torch.float64, device="cuda")
        tv = t_v.contiguous()
        _lib.check(load().tc_clustering(self._h, ctypes.c_void_p(tv.data_ptr()), ctypes.c_void_p(cc.data_ptr()),
                                        _stream(stream)), "tc_clustering")
        return cc[:n]

    def count_ex(self, options: _lib.Options | None = None, trace_cap: int = 0, busy: bool = False, stream=None,
                 timing: bool = False, streamed: bool = False):
        """Count with explicit options; optionally record the schedule.

        Returns (T, meta, chunks, busy): chunks is an int64 CUDA tensor of shape (k, 5)
        holding (class, cost_lo, cost_hi, task_lo, task_hi) per chunk taken, costs counted
        within the class; busy is (W_small + W_big, 2): clock cycles and chunks per worker.
        """
        torch = _torch()
        tr = _lib.CountTrace()
        ch = bz = None
        if trace_cap > 0:
            ch = torch.zeros(4 * trace_cap, dtype=torch.int64, device="cuda")
            tr.chunks = ch.data_ptr()
            tr.cap = trace_cap
        if busy:
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            # small-class warps (at most 64 resident per SM) plus big-class blocks (at most 32 per SM)
            bz = torch.zeros(2 * sms * 96, dtype=torch.int64, device="cuda")
            tr.workers_busy = bz.data_ptr()
        tr.count_streamed = 1 if streamed else 0
        t = ctypes.c_uint64()
        opt = ctypes.byref(options) if options is not None else None
        use_trace = trace_cap > 0 or busy or timing or streamed
        _lib.check(load().tc_count_ex(self._h, opt, _stream(stream), ctypes.byref(t),
                                      ctypes.byref(tr) if use_trace else None), "tc_count_ex")
        meta = {"n_chunks": tr.n_chunks, "n_workers": list(tr.n_workers), "total_cost": list(tr.total_cost),
                "min_chunk": list(tr.min_chunk), "tasks_small": tr.tasks_small, "prefix_ms": tr.prefix_ms,
                "kernel_small_ms": tr.kernel_small_ms, "kernel_big_ms": tr.kernel_big_ms,
                "kernel_ms": tr.kernel_small_ms + tr.kernel_big_ms, "streamed": list(tr.streamed)}
        chunks = None
        if ch is not None:
            raw = ch.view(-1, 4)[:min(tr.n_chunks, trace_cap)]
            cls = torch.bitwise_right_shift(raw[:, 0], 56)
            lo = torch.bitwise_and(raw[:, 0], (1 << 56) - 1)
            chunks = torch.stack([cls, lo, raw[:, 1], raw[:, 2], raw[:, 3]], dim=1)
        busy_t = bz.view(-1, 2)[:tr.n_workers[0] + tr.n_workers[1]] if bz is not None else None
        return int(t.value), meta, chunks, busy_t

    def vertex_cost(self, fn: int, stream=None):
        """Per-vertex cost f(v) as an int64 CUDA tensor (values < 2^63)."""
        torch = _torch()
        n = self.info()["n"]
        f = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        _lib.check(load().tc_vertex_cost(self._h, int(fn), _stream(stream), ctypes.c_void_p(f.data_ptr())),
                   "tc_vertex_cost")
        return f[:n]

    # ------------------------------------------------------------------ introspection
    def info(self) -> dict:
        gi = _lib.GraphInfo()
        _lib.check(load().tc_graph_get_info(self._h, ctypes.byref(gi)), "tc_graph_get_info")
        return gi.as_dict()

    def csr(self):
        """Clones of (deg int32[n], off int64[n+1], cols int32[m_hat], tasks int32[T, 4])."""
        info = self.info()
        d, o, c, t = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
        _lib.check(load().tc_graph_csr(self._h, ctypes.byref(d), ctypes.byref(o), ctypes.byref(c), ctypes.byref(t)),
                   "tc_graph_csr")
        n, mh, T = info["n"], info["m_hat"], info["tasks"]
        deg = _view(d.value, n, "<i4").clone()
        off = _view(o.value, n + 1, "<i8").clone()
        cols = _view(c.value, mh, "<i4").clone()
        tasks = _view(t.value, 4 * T, "<i4").clone().view(-1, 4)
        return deg, off, cols, tasks


def count_graphs(graphs, stream=None) -> list:
    """Totals of several built graphs, counted back to back with one synchronisation."""
    k = len(graphs)
    hs = (ctypes.c_void_p * max(k, 1))(*[g.handle for g in graphs])
    totals = (ctypes.c_uint64 * max(k, 1))()
    _lib.check(load().tc_count_graphs(hs, k, _stream(stream), totals), "tc_count_graphs")
    return [int(totals[j]) for j in range(k)]


def _array_ptr(a, dtype_name: str):
    """(pointer, length, keepalive) of a numpy array or torch tensor (host, pinned host or CUDA)."""
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != getattr(torch, dtype_name):
                raise TypeError(f"expected a {dtype_name} tensor")
            t = a.contiguous()
            return ctypes.c_void_p(t.data_ptr()), int(t.numel()), t
    except ImportError:  # pragma: no cover
        pass
    import numpy as np
    x = np.ascontiguousarray(a, dtype=getattr(np, dtype_name))
    return x.ctypes.data_as(ctypes.c_void_p), int(x.size), x


def surrogate_plan(off, cols, nparts: int = 0, part_bytes: int = 0, fn: int = TC_FN_NEW,
                   max_parts: int = _lib.TC_SURROGATE_MAX_PARTS, stream=None):
    """Cuts (int32 numpy array of P + 1 vertex ids) of Sec. IV-B's cost-balanced non-overlapping
    partition of the oriented lists (off, cols) under the per-vertex cost `fn` (TC_FN_NEW: equal
    work, Sec. IV-F; TC_FN_LIST: equal list entries).  nparts > 0 fixes P; nparts = 0 picks the
    smallest P whose parts' list slices each fit in part_bytes."""
    import numpy as np
    op, n1, ko = _array_ptr(off, "int64")
    cp, m, kc = _array_ptr(cols, "int32")
    cap = (nparts if nparts > 0 else max_parts) + 1
    cuts = np.zeros(cap, np.int32)
    P = ctypes.c_int32()
    rc = load().tc_surrogate_plan(op, cp, n1 - 1, m, int(fn), int(nparts), int(part_bytes), int(max_parts),
                                  _stream(stream), cuts.ctypes.data_as(ctypes.c_void_p), ctypes.byref(P))
    del ko, kc
    _lib.check(rc, "tc_surrogate_plan")
    return cuts[:P.value + 1].copy()


def surrogate_plan_both(off, cols, work_parts: int, part_bytes: int, fn: int = TC_FN_NEW,
                        max_parts: int = _lib.TC_SURROGATE_MAX_PARTS, stream=None):
    """Cuts (int32 numpy array of P + 1 vertex ids) bounded in work and size at once: the union of
    the cuts of `work_parts` parts of equal cost `fn` and of the fewest equal-size parts whose list
    slices each fit in part_bytes."""
    import numpy as np
    op, n1, ko = _array_ptr(off, "int64")
    cp, m, kc = _array_ptr(cols, "int32")
    cuts = np.zeros(int(work_parts) + int(max_parts) + 1, np.int32)
    P = ctypes.c_int32()
    rc = load().tc_surrogate_plan_both(op, cp, n1 - 1, m, int(fn), int(work_parts), int(part_bytes), int(max_parts),
                                       _stream(stream), cuts.ctypes.data_as(ctypes.c_void_p), ctypes.byref(P))
    del ko, kc
    _lib.check(rc, "tc_surrogate_plan_both")
    return cuts[:P.value + 1].copy()


def count_surrogate(off, cols, cuts, part_lo: int = 0, part_hi: int | None = None,
                    options: _lib.Options | None = None, stream=None, stats: bool = False):
    """(total, table) of the count over the non-overlapping partition `cuts` (Sec. IV):
    table[i, j] sums SurrogateCount(N_v, j) over v in V_i, for the receiving parts
    part_lo <= j < part_hi (all parts by default); total is the table's sum.  With stats=True a
    third element holds the work done (items, staged and streamed entries, copied bytes, kernel
    times)."""
    import numpy as np
    op, n1, ko = _array_ptr(off, "int64")
    cp, m, kc = _array_ptr(cols, "int32")
    cu = np.ascontiguousarray(cuts, dtype=np.int32)
    P = len(cu) - 1
    hi = P if part_hi is None else int(part_hi)
    table = np.zeros(max(P, 1) * max(P, 1), np.uint64)
    t = ctypes.c_uint64()
    opt = ctypes.byref(options) if options is not None else None
    st = _lib.SurrogateStats()
    rc = load().tc_count_surrogate(op, cp if m else None, n1 - 1, m, cu.ctypes.data_as(ctypes.c_void_p), P,
                                   int(part_lo), hi, opt, _stream(stream), table.ctypes.data_as(ctypes.c_void_p),
                                   ctypes.byref(t), ctypes.byref(st) if stats else None)
    del ko, kc
    _lib.check(rc, "tc_count_surrogate")
    if stats:
        return int(t.value), table[:P * P].reshape(P, P), st.as_dict()
    return int(t.value), table[:P * P].reshape(P, P)


from .batch import Batch, autotune  # noqa: E402
from .server import Server  # noqa: E402
