"""Request loop with continuous batching (binding of the tc_server_* calls)."""
from __future__ import annotations

import ctypes

from . import _lib


class Server:
    def __init__(self, hbm_budget_bytes: int, slots: int = 4, options=None):
        from . import load
        h = ctypes.c_void_p()
        opt = ctypes.byref(options) if options is not None else None
        _lib.check(load().tc_server_create(int(hbm_budget_bytes), int(slots), opt, ctypes.byref(h)),
                   "tc_server_create")
        self._h = h
