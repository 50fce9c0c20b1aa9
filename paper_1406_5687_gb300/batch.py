"""Batched counting: binding of the tc_batch_* calls (argument marshalling only).

Many independent graphs are packed into disjoint unions, built by one pass of the
single-graph pipeline per pack and counted by one replayed CUDA graph; each graph
keeps its own exact total.  Every step runs in the CUDA library.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib


def _lists(graphs):
    """Pointer tables and sizes for a list of (src, dst, n) with numpy or torch int32 edges."""
    from . import _edge_ptrs
    k = len(graphs)
    srcs = (ctypes.c_void_p * max(k, 1))()
    dsts = (ctypes.c_void_p * max(k, 1))()
    m = np.zeros(max(k, 1), np.int64)
    n = np.zeros(max(k, 1), np.int32)
    keep = []
    for j, (s, d, nj) in enumerate(graphs):
        sp, dp, mj, kp = _edge_ptrs(s, d)
        srcs[j], dsts[j] = sp.value, dp.value
        m[j], n[j] = mj, int(nj)
        keep.append(kp)
    return srcs, dsts, m, n, keep


class Batch:
    """k graphs built into packs and counted together.

    ``graphs`` is a sequence of ``(src, dst, n)`` with int32 numpy arrays (host) or
    int32 torch tensors (host or CUDA)."""

    def __init__(self, handle, k):
        self._h = handle
        self.k = k

    @classmethod
    def build(cls, graphs, options=None, pack_edges: int = 0, stream=None) -> "Batch":
        from . import _stream, load
        graphs = list(graphs)
        srcs, dsts, m, n, keep = _lists(graphs)
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        rc = load().tc_batch_build(srcs, dsts, m.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                   len(graphs), int(pack_edges), opt, _stream(stream), ctypes.byref(h))
        del keep
        _lib.check(rc, "tc_batch_build")
        return cls(h, len(graphs))

    def run(self, totals_dev, stream=None):
        """Enqueue the count of every graph into totals_dev (torch int64 CUDA tensor of k)."""
        from . import _stream, load
        if totals_dev.numel() < self.k:
            raise ValueError("totals_dev holds fewer than k entries")
        _lib.check(load().tc_batch_run(self._h, _stream(stream), ctypes.c_void_p(totals_dev.data_ptr())),
                   "tc_batch_run")

    def check(self, stream=None):
        from . import _stream, load
        _lib.check(load().tc_batch_check(self._h, _stream(stream)), "tc_batch_check")

    def count(self, stream=None) -> np.ndarray:
        """Exact totals of all graphs (uint64, host)."""
        from . import _stream, load
        out = np.zeros(max(self.k, 1), np.uint64)
        _lib.check(load().tc_batch_count(self._h, _stream(stream), out.ctypes.data_as(ctypes.c_void_p)),
                   "tc_batch_count")
        return out[:self.k]

    def info(self) -> dict:
        from . import load
        bi = _lib.BatchInfo()
        _lib.check(load().tc_batch_get_info(self._h, ctypes.byref(bi)), "tc_batch_get_info")
        return bi.as_dict()

    def graph_edges(self) -> np.ndarray:
        """Distinct edges of each graph (int64, host)."""
        from . import load
        out = np.zeros(max(self.k, 1), np.int64)
        _lib.check(load().tc_batch_graph_edges(self._h, out.ctypes.data_as(ctypes.c_void_p)), "tc_batch_graph_edges")
        return out[:self.k]

    def set_options(self, options):
        from . import load
        _lib.check(load().tc_batch_set_options(self._h, ctypes.byref(options)), "tc_batch_set_options")

    def free(self):
        from . import load
        if self._h:
            load().tc_batch_free(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


_TUNED_FIELDS = ("small_max", "warps_per_block", "big_warps", "piece", "static_percent")


def workload_signature(graphs) -> str:
    """Key of a tuning result: the device and log2 buckets of the workload's shape (graph
    count, mean input edges, mean vertices)."""
    import math
    import torch
    from . import _edge_ptrs
    k = len(graphs)
    m = [int(_edge_ptrs(s, d)[2]) for s, d, _ in graphs]
    n = [int(nj) for _, _, nj in graphs]
    b = lambda x: int(round(math.log2(max(x, 1))))  # noqa: E731
    dev = torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "none"
    return f"{dev}|k{b(k)}|m{b(sum(m) / max(k, 1))}|n{b(sum(n) / max(k, 1))}"


def autotune(graphs, options=None, reps: int = 3, stream=None, cap: int = 64, cache_path=None):
    """Time the batched count of `graphs` over the library's grid of hub thresholds and
    launch shapes.  Returns (best Options, report dict with every candidate's time).

    With cache_path, a result tuned before for the same device and workload shape (see
    workload_signature) is read from that JSON file instead, and new results are added."""
    import json
    import os
    from . import _stream, default_options, load
    graphs = list(graphs)
    sig = workload_signature(graphs) if cache_path else None
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
        if sig in cache:
            base = options if options is not None else default_options()
            best = _lib.Options()
            ctypes.memmove(ctypes.byref(best), ctypes.byref(base), ctypes.sizeof(best))
            for k in _TUNED_FIELDS:
                setattr(best, k, int(cache[sig][k]))
            return best, {"cached": True, "signature": sig, **cache[sig]}
    srcs, dsts, m, n, keep = _lists(graphs)
    best = _lib.Options()
    entries = (_lib.TuneEntry * cap)()
    rep = _lib.TuneReport(entries, cap, 0, -1.0, -1.0)
    opt = ctypes.byref(options) if options is not None else None
    rc = load().tc_batch_autotune(srcs, dsts, m.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                                  len(graphs), opt, int(reps), _stream(stream), ctypes.byref(best), ctypes.byref(rep))
    del keep
    _lib.check(rc, "tc_batch_autotune")
    cands = [{"small_max": e.small_max, "warps_per_block": e.warps_per_block, "big_warps": e.big_warps,
              "piece": e.piece, "static_percent": e.static_percent, "ms": e.ms} for e in entries[:min(rep.n, cap)]]
    report = {"cached": False, "tried": rep.n, "best_ms": rep.best_ms, "default_ms": rep.default_ms,
              "candidates": cands}
    if cache_path:
        cache = {}
        if os.path.exists(cache_path):
            with open(cache_path) as f:
                cache = json.load(f)
        cache[sig] = {**{k: getattr(best, k) for k in _TUNED_FIELDS}, "best_ms": rep.best_ms}
        tmp = f"{cache_path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
        report["signature"] = sig
    return best, report
