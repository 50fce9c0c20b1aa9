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
    lib.tc_free(None)
