"""ctypes binding of the C ABI in ``include/tc.h`` (argument marshalling only).

Every step of the count runs in the CUDA library ``libtcgb300.so``; this module
only converts Python / numpy / torch arguments into pointers and sizes.  If the
library cannot be built or loaded, importing the functions raises: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_lock = threading.Lock()

TC_OK = 0
STATUS_NAMES = {0: "TC_OK", 1: "TC_ERR_INVALID_ARG", 2: "TC_ERR_VERTEX_RANGE", 3: "TC_ERR_OOM",
                4: "TC_ERR_CUDA", 5: "TC_ERR_TIMEOUT", 6: "TC_ERR_BUDGET", 7: "TC_ERR_UNSUPPORTED",
                8: "TC_ERR_CANCELLED"}
(TC_ERR_INVALID_ARG, TC_ERR_VERTEX_RANGE, TC_ERR_OOM, TC_ERR_CUDA, TC_ERR_TIMEOUT, TC_ERR_BUDGET,
 TC_ERR_UNSUPPORTED, TC_ERR_CANCELLED) = range(1, 9)
TC_COST_EDGE, TC_COST_MERGE, TC_COST_ONE, TC_COST_DEGREE, TC_COST_PATRIC, TC_COST_NEW = range(6)
TC_FN_ONE, TC_FN_DEGREE, TC_FN_PATRIC, TC_FN_NEW, TC_FN_LIST = range(5)
TC_INPUT_SANITIZE, TC_INPUT_STRICT = 0, 1
TC_COUNT_STATIC_MAX_TASKS = 1 << 19  # include/tc.h
TC_TRIM_MIN_ENTRIES = 16  # include/tc.h
TC_SURROGATE_MAX_PARTS = 1024  # include/tc.h
TC_SURROGATE_PIECE = 256  # include/tc.h

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
RELEASE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)


class TcError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}")
        self.code = code


class Options(ctypes.Structure):
    _fields_ = [("input_policy", ctypes.c_int32), ("cost_model", ctypes.c_int32), ("piece", ctypes.c_int32),
                ("warps_per_block", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("big_warps", ctypes.c_int32), ("small_max", ctypes.c_int32),
                ("static_percent", ctypes.c_int32), ("min_chunk", ctypes.c_int64), ("c_task", ctypes.c_int32),
                ("c_owner", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("retry_limit", ctypes.c_int64),
                ("alloc", ALLOC_FN), ("release", RELEASE_FN), ("alloc_ctx", ctypes.c_void_p)]


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("max_degree", ctypes.c_int32), ("max_dhat", ctypes.c_int32),
                ("id_bits", ctypes.c_int32), ("m_in", ctypes.c_int64), ("self_loops", ctypes.c_int64),
                ("duplicates", ctypes.c_int64), ("m_hat", ctypes.c_int64), ("tasks", ctypes.c_int64),
                ("tasks_small", ctypes.c_int64),
                ("sum_dhat_v", ctypes.c_uint64), ("sum_dhat_u", ctypes.c_uint64), ("sum_stream", ctypes.c_uint64),
                ("device_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CountTrace(ctypes.Structure):
    _fields_ = [("chunks", ctypes.c_void_p), ("cap", ctypes.c_int64), ("workers_busy", ctypes.c_void_p),
                ("n_chunks", ctypes.c_int64), ("n_workers", ctypes.c_int64 * 2), ("total_cost", ctypes.c_uint64 * 2),
                ("min_chunk", ctypes.c_uint64 * 2), ("tasks_small", ctypes.c_int64), ("prefix_ms", ctypes.c_float),
                ("kernel_small_ms", ctypes.c_float), ("kernel_big_ms", ctypes.c_float),
                ("count_streamed", ctypes.c_int32), ("streamed", ctypes.c_int64 * 2)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("packs", ctypes.c_int32), ("max_dhat", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("m_in", ctypes.c_int64), ("m_hat", ctypes.c_int64),
                ("tasks", ctypes.c_int64), ("tasks_small", ctypes.c_int64), ("device_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class TuneEntry(ctypes.Structure):
    _fields_ = [("small_max", ctypes.c_int32), ("warps_per_block", ctypes.c_int32), ("big_warps", ctypes.c_int32),
                ("piece", ctypes.c_int32), ("static_percent", ctypes.c_int32), ("ms", ctypes.c_float)]


class TuneReport(ctypes.Structure):
    _fields_ = [("entries", ctypes.POINTER(TuneEntry)), ("cap", ctypes.c_int32), ("n", ctypes.c_int32),
                ("best_ms", ctypes.c_float), ("default_ms", ctypes.c_float)]


class SurrogateStats(ctypes.Structure):
    _fields_ = [("items", ctypes.c_int64), ("staged", ctypes.c_int64), ("streamed", ctypes.c_int64),
                ("copied_bytes", ctypes.c_int64), ("route_ms", ctypes.c_float), ("count_ms", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_uint64), ("total", ctypes.c_uint64), ("status", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("group", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double), ("t_done", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("finished", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("groups", ctypes.c_int64), ("grouped", ctypes.c_int64), ("bytes_in_flight", ctypes.c_int64),
                ("peak_bytes_in_flight", ctypes.c_int64), ("peak_slots_busy", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


# name -> (restype, argtypes); every function declared in include/tc.h
P = ctypes.c_void_p
SIGNATURES = {
    "tc_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tc_version": (ctypes.c_char_p, []),
    "tc_options_default": (None, [ctypes.POINTER(Options)]),
    "tc_build": (ctypes.c_int, [P, P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Options), P, ctypes.POINTER(P)]),
    "tc_build_pairs": (ctypes.c_int, [P, ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(Options), P,
                                      ctypes.POINTER(P)]),
    "tc_count_graphs": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int32, P, P]),
    "tc_free": (None, [P]),
    "tc_count": (ctypes.c_int, [P, P, ctypes.POINTER(ctypes.c_uint64)]),
    "tc_count_async": (ctypes.c_int, [P, P, P]),
    "tc_count_partition": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P, ctypes.POINTER(ctypes.c_uint64)]),
    "tc_graph_check": (ctypes.c_int, [P, P]),
    "tc_count_per_vertex": (ctypes.c_int, [P, P, P, ctypes.POINTER(ctypes.c_uint64)]),
    "tc_count_per_edge": (ctypes.c_int, [P, P, P, ctypes.POINTER(ctypes.c_uint64)]),
    "tc_clustering": (ctypes.c_int, [P, P, P, P]),
    "tc_graph_get_info": (ctypes.c_int, [P, ctypes.POINTER(GraphInfo)]),
    "tc_graph_csr": (ctypes.c_int, [P, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P)]),
    "tc_vertex_cost": (ctypes.c_int, [P, ctypes.c_int32, P, P]),
    "tc_count_ex": (ctypes.c_int, [P, ctypes.POINTER(Options), P, ctypes.POINTER(ctypes.c_uint64),
                                   ctypes.POINTER(CountTrace)]),
    "tc_kernel_launches": (ctypes.c_int64, []),
    "tc_count_static": (ctypes.c_int, [P, P, P]),
    "tc_wait_selftest": (ctypes.c_int, [ctypes.c_int64, P]),
    "tc_count_surrogate": (ctypes.c_int, [P, P, ctypes.c_int32, ctypes.c_int64, P, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, ctypes.POINTER(Options), P, P,
                                          ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(SurrogateStats)]),
    "tc_surrogate_plan": (ctypes.c_int, [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.c_int64, ctypes.c_int32, P, P, ctypes.POINTER(ctypes.c_int32)]),
    "tc_surrogate_plan_both": (ctypes.c_int, [P, P, ctypes.c_int32, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int64, ctypes.c_int32, P, P, ctypes.POINTER(ctypes.c_int32)]),
    "tc_batch_build": (ctypes.c_int, [P, P, P, P, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(Options), P,
                                      ctypes.POINTER(P)]),
    "tc_batch_run": (ctypes.c_int, [P, P, P]),
    "tc_batch_check": (ctypes.c_int, [P, P]),
    "tc_batch_count": (ctypes.c_int, [P, P, P]),
    "tc_batch_get_info": (ctypes.c_int, [P, ctypes.POINTER(BatchInfo)]),
    "tc_batch_graph_edges": (ctypes.c_int, [P, P]),
    "tc_batch_set_options": (ctypes.c_int, [P, ctypes.POINTER(Options)]),
    "tc_batch_free": (None, [P]),
    "tc_batch_autotune": (ctypes.c_int, [P, P, P, P, ctypes.c_int32, ctypes.POINTER(Options), ctypes.c_int32, P,
                                         ctypes.POINTER(Options), ctypes.POINTER(TuneReport)]),
    "tc_server_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(Options),
                                        ctypes.POINTER(P)]),
    "tc_server_submit": (ctypes.c_int, [P, P, P, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64]),
    "tc_server_poll": (ctypes.c_int, [P, ctypes.POINTER(Result), ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "tc_server_cancel": (ctypes.c_int, [P, ctypes.c_uint64, ctypes.POINTER(ctypes.c_int64)]),
    "tc_server_drain": (ctypes.c_int, [P, ctypes.c_int64]),
    "tc_server_get_stats": (ctypes.c_int, [P, ctypes.POINTER(ServerStats)]),
    "tc_server_destroy": (None, [P]),
}


def library_path() -> str:
    return os.path.join(_HERE, "libtcgb300.so")


def load(build_if_missing: bool = True):
    """Load (building first if needed) the CUDA library; raises if it cannot."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing:
                from . import build as _build
                _build.build()
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path}")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(code: int, where: str):
    if code != TC_OK:
        raise TcError(code, where)


def default_options(**kw) -> Options:
    o = Options()
    load().tc_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise AttributeError(k)
        setattr(o, k, v)
    return o
