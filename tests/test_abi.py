"""The C-ABI library loads and exports every function include/tc.h declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "tc.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z_0-9]*\s*\**\s+\**\s*(tc_[a-z_0-9]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["tc_build", "tc_count", "tc_count_per_vertex", "tc_graph_get_info", "tc_free",
                     "tc_status_str", "tc_batch_count", "tc_server_create", "tc_server_submit",
                     "tc_server_poll", "tc_server_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1406_5687_gb300 import _lib
    lib = _lib.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name


def test_host_only_calls():
    from paper_1406_5687_gb300 import _lib
    lib = _lib.load()
    assert lib.tc_status_str(0) == b"ok"
    assert lib.tc_status_str(2).startswith(b"vertex id")
    assert b"sm_103a" in lib.tc_version()
    o = _lib.default_options()
    assert (o.piece, o.warps_per_block, o.big_warps, o.small_max, o.static_percent, o.cost_model) == \
        (2048, 16, 16, 64, 50, 0)
    # argument checks that return before touching a device
    h = ctypes.c_void_p()
    assert lib.tc_build(None, None, -1, 10, None, None, ctypes.byref(h)) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_build(None, None, 5, 10, None, None, ctypes.byref(h)) == _lib.TC_ERR_INVALID_ARG
    for bad in (_lib.default_options(piece=1000), _lib.default_options(small_max=100),
                _lib.default_options(big_warps=32), _lib.default_options(static_percent=101)):
        assert lib.tc_build(None, None, 0, 10, ctypes.byref(bad), None, ctypes.byref(h)) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_count(None, None, None) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_build_pairs(None, 5, 10, None, None, ctypes.byref(h)) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_build_pairs(None, -1, 10, None, None, ctypes.byref(h)) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_count_graphs(None, -1, None, None) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_count_graphs(None, 2, None, None) == _lib.TC_ERR_INVALID_ARG
    lib.tc_free(None)


def test_surrogate_argument_checks():
    """Bad sizes, ranges and cuts are refused before any device work."""
    import numpy as np
    from paper_1406_5687_gb300 import _lib
    lib = _lib.load()
    off = np.zeros(11, np.int64)
    t = ctypes.c_uint64()
    P = ctypes.c_int32()
    o = off.ctypes.data_as(ctypes.c_void_p)

    def count(cuts, lo=0, hi=None, n=10, m=0):
        c = np.asarray(cuts, np.int32)
        return lib.tc_count_surrogate(o, None, n, m, c.ctypes.data_as(ctypes.c_void_p), len(c) - 1, lo,
                                      len(c) - 1 if hi is None else hi, None, None, None, ctypes.byref(t), None)

    for cuts in ([1, 10], [0, 9], [0, 6, 5, 10], [0]):
        assert count(cuts) == _lib.TC_ERR_INVALID_ARG, cuts
    assert count([0, 5, 10], lo=1, hi=0) == _lib.TC_ERR_INVALID_ARG
    assert count([0, 5, 10], lo=0, hi=3) == _lib.TC_ERR_INVALID_ARG
    assert count([0, 10], n=-1) == _lib.TC_ERR_INVALID_ARG
    assert count([0, 10], m=5) == _lib.TC_ERR_INVALID_ARG  # entries but no cols
    too_many = np.linspace(0, 10, _lib.TC_SURROGATE_MAX_PARTS + 2).astype(np.int32)
    assert count(too_many) == _lib.TC_ERR_INVALID_ARG
    cuts = np.zeros(8, np.int32)
    cp = cuts.ctypes.data_as(ctypes.c_void_p)
    # nparts = 0 needs a part size; negative sizes are refused
    new = _lib.TC_FN_NEW
    assert lib.tc_surrogate_plan(o, None, 10, 0, new, 0, 0, 7, None, cp, ctypes.byref(P)) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_surrogate_plan(o, None, 10, 0, new, 2, -1, 7, None, cp, ctypes.byref(P)) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_surrogate_plan(o, None, 10, 0, new, _lib.TC_SURROGATE_MAX_PARTS + 1, 0, 7, None, cp,
                                 ctypes.byref(P)) == _lib.TC_ERR_INVALID_ARG
    for fn in (-1, _lib.TC_FN_LIST + 1):
        assert lib.tc_surrogate_plan(o, None, 10, 0, fn, 2, 0, 7, None, cp, ctypes.byref(P)) == _lib.TC_ERR_INVALID_ARG


def test_header_compiles_as_c_and_links():
    """include/tc.h as plain C11 against the shared library, with the calls that need no device."""
    import shutil
    import subprocess
    import tempfile
    from paper_1406_5687_gb300 import _lib
    _lib.load()
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc is not installed")
    libdir = os.path.dirname(_lib.library_path())
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "abi_from_c")
        cmd = [gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
               os.path.join(ROOT, "tests", "native", "abi_from_c.c"), "-L", libdir, "-ltcgb300",
               "-Wl,-rpath," + libdir, "-o", exe]
        build = subprocess.run(cmd, capture_output=True, text=True)
        assert build.returncode == 0, build.stderr
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "abi from C: ok" in r.stdout
