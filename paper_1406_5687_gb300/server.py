"""Serving with continuous batching: binding of the tc_server_* calls (marshalling only).

The server borrows each request's edge arrays until its result is polled; this binding
keeps a reference to them until then, so callers need not.
"""
from __future__ import annotations

import ctypes
import itertools
import threading

from . import _lib


class Server:
    """Slot threads of the CUDA library that admit queued graphs by a device-memory budget,
    count them alone or grouped into one batch pack, and overlap on the GPU."""

    def __init__(self, hbm_budget_bytes: int, slots: int = 4, group_edges: int = 0, options=None):
        from . import load
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        _lib.check(load().tc_server_create(int(hbm_budget_bytes), int(slots), int(group_edges), opt,
                                           ctypes.byref(h)), "tc_server_create")
        self._h = h
        self._ids = itertools.count()
        self._pending = {}   # internal id -> (caller's tag, arrays kept alive)
        self._lock = threading.Lock()

    def submit(self, src, dst, n: int, tag=None) -> int:
        """Queue one graph (numpy or torch int32 arrays, host or CUDA); returns its id."""
        from . import _edge_ptrs, load
        sp, dp, m, keep = _edge_ptrs(src, dst)
        rid = next(self._ids)
        with self._lock:
            self._pending[rid] = (rid if tag is None else tag, keep)
        rc = load().tc_server_submit(self._h, sp, dp, m, int(n), rid)
        if rc != _lib.TC_OK:
            with self._lock:
                self._pending.pop(rid, None)
            _lib.check(rc, "tc_server_submit")
        return rid

    def cancel(self, tag) -> int:
        """Withdraw the still-queued requests submitted with `tag`; returns how many.  Their
        results come back from poll with status TC_ERR_CANCELLED."""
        from . import load
        with self._lock:
            rids = [rid for rid, (t, _) in self._pending.items() if t == tag]
        n = 0
        for rid in rids:
            k = ctypes.c_int64()
            _lib.check(load().tc_server_cancel(self._h, rid, ctypes.byref(k)), "tc_server_cancel")
            n += k.value
        return n

    def poll(self, max_results: int = 1024) -> list[dict]:
        from . import load
        buf = (_lib.Result * max(1, max_results))()
        k = ctypes.c_int32()
        _lib.check(load().tc_server_poll(self._h, buf, max_results, ctypes.byref(k)), "tc_server_poll")
        out = []
        with self._lock:
            for r in buf[:k.value]:
                tag, _ = self._pending.pop(r.tag, (r.tag, None))
                out.append({"id": r.tag, "tag": tag, "total": int(r.total), "status": r.status, "slot": r.slot,
                            "group": r.group, "t_submit": r.t_submit, "t_start": r.t_start, "t_done": r.t_done})
        return out

    def drain(self, timeout_ms: int = -1):
        from . import load
        _lib.check(load().tc_server_drain(self._h, int(timeout_ms)), "tc_server_drain")

    def stats(self) -> dict:
        from . import load
        st = _lib.ServerStats()
        _lib.check(load().tc_server_get_stats(self._h, ctypes.byref(st)), "tc_server_get_stats")
        return st.as_dict()

    def close(self):
        from . import load
        if self._h:
            load().tc_server_destroy(self._h)
            self._h = None
            with self._lock:
                self._pending.clear()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
