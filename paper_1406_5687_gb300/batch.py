"""Batched counting over many built graphs (binding of the tc_batch_* calls)."""
from __future__ import annotations

import ctypes

from . import _lib


class Batch:
    """k graphs counted by one persistent launch replayed from a captured CUDA graph."""

    def __init__(self, graphs, options=None, stream=None):
        from . import _stream, load
        self._graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self._graphs))(*[g.handle for g in self._graphs])
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        _lib.check(load().tc_batch_create(arr, len(self._graphs), opt, _stream(stream), ctypes.byref(h)),
                   "tc_batch_create")
        self._h = h

    def run(self, out, stream=None):
        from . import _stream, load
        _lib.check(load().tc_batch_run(self._h, _stream(stream), ctypes.c_void_p(out.data_ptr())), "tc_batch_run")

    def free(self):
        from . import load
        if self._h:
            load().tc_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
