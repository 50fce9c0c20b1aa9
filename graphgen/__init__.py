"""Seeded synthetic graph inputs (COO edge lists of int32 vertex ids).

This package only makes inputs.  It holds none of the triangle-counting
arithmetic and is imported by both the CPU oracle's tests and the GPU path's
tests and benchmark, so both sides count the same graphs.

The random generators live in ``graphgen.c`` (counter-based SplitMix64 draws,
so each graph depends only on its seed); the small closed-form families are
in :mod:`graphgen.families`; the named workloads (the Erdos-Renyi, Barabasi-
Albert, Chung-Lu, batched and serving recipes) are in
:mod:`graphgen.workloads`.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB_PATH = os.path.join(_HERE, "libgraphgen.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to its source (gcc, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
            lib.gg_er.restype = ctypes.c_int64
            lib.gg_ba.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, i32p, i32p]
            lib.gg_ba.restype = ctypes.c_int64
            lib.gg_chung_lu.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int64, ctypes.c_uint64, i32p, i32p]
            lib.gg_chung_lu.restype = ctypes.c_int64
            lib.gg_chung_lu_weights.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                                ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
            lib.gg_chung_lu_weights.restype = ctypes.c_int
            lib.gg_key.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_key.restype = ctypes.c_uint64
            lib.gg_draw.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_draw.restype = ctypes.c_uint64
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def erdos_renyi(n: int, m: int, seed: int):
    """G(n, m): ``m`` distinct undirected non-loop pairs, uniform; returns (src, dst) int32."""
    lib = _load()
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = lib.gg_er(n, m, seed, _ptr(src), _ptr(dst))
    if rc != m:
        raise ValueError(f"gg_er(n={n}, m={m}) failed with {rc}")
    return src, dst


def barabasi_albert(n: int, k: int, seed: int):
    """Preferential attachment with ``k`` distinct targets per new vertex; m = k(n-k)."""
    lib = _load()
    m = k * (n - k)
    src = np.empty(m, dtype=np.int32)
    dst = np.empty(m, dtype=np.int32)
    rc = lib.gg_ba(n, k, seed, _ptr(src), _ptr(dst))
    if rc != m:
        raise ValueError(f"gg_ba(n={n}, k={k}) failed with {rc}")
    return src, dst


def chung_lu(n: int, gamma: float, avg_deg: float, w_max: float, draws: int, seed: int):
    """Chung-Lu edge draws (self-loops and repeats kept); returns (src, dst) int32."""
    lib = _load()
    src = np.empty(draws, dtype=np.int32)
    dst = np.empty(draws, dtype=np.int32)
    rc = lib.gg_chung_lu(n, float(gamma), float(avg_deg), float(w_max), draws, seed, _ptr(src), _ptr(dst))
    if rc != draws:
        raise ValueError(f"gg_chung_lu failed with {rc}")
    return src, dst


def chung_lu_weights(n: int, gamma: float, avg_deg: float, w_max: float) -> np.ndarray:
    lib = _load()
    w = np.empty(n, dtype=np.float64)
    rc = lib.gg_chung_lu_weights(n, float(gamma), float(avg_deg), float(w_max),
                                 w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if rc != 0:
        raise ValueError("bad Chung-Lu parameters")
    return w


def draw(seed: int, tag: int, i: int) -> int:
    """Draw ``i`` of the counter-based stream (seed, tag): a uint64."""
    lib = _load()
    return int(lib.gg_draw(lib.gg_key(seed, tag), i))
