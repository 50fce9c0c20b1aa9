"""tc_count_static: counting with no device allocation, against the oracle and tc_count.

Some callers cannot allocate device memory when they count -- their memory is owned
by their own pool, or an allocation there could block or is not allowed.  For them
the library offers tc_count_static, which keeps the count's scratch in a fixed device
array declared by the library.  This file checks, through the C ABI, that two calls in
a row give the oracle's exact total and the same total as tc_count (tolerance 0: counts
are integers), that graphs with too many tasks are refused, and that the call takes no
memory through the graph's allocator.  It is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import graphgen  # noqa: E402
import oracle  # noqa: E402
import paper_1406_5687_gb300 as tc  # noqa: E402
from graphgen import families as F  # noqa: E402
from paper_1406_5687_gb300 import _lib  # noqa: E402


def _graphs():
    n = 200000
    s, d = graphgen.chung_lu(n, 2.1, 4.0, 3000.0, 400_000, 31)
    yield "chung_lu_200k", n, s, d
    n, s, d = F.wheel(5000)
    yield "wheel_5000", n, s, d
    n = 3000
    s, d = graphgen.chung_lu(n, 2.05, 100.0, 1500.0, 150_000, 32)
    yield "chung_lu_dense", n, s, d
    yield "no_edges", 10, np.zeros(0, np.int32), np.zeros(0, np.int32)
    # K_200: its lists hold 199, 198, ..., 0 entries, so owners fall in both task classes
    n, s, d = F.complete(200)
    yield "complete_200", n, s, d


CASES = 5


def _static_count(lib, g, out, stream):
    rc = lib.tc_count_static(g.handle, ctypes.c_void_p(stream.cuda_stream), ctypes.c_void_p(out.data_ptr()))
    assert rc == _lib.TC_OK, _lib.STATUS_NAMES.get(rc, rc)
    stream.synchronize()
    return int(out.item())


@pytest.mark.parametrize("case", list(range(CASES)))
def test_two_calls_match_the_oracle_and_tc_count(case):
    name, n, s, d = list(_graphs())[case]
    want = oracle.count_edges(n, s, d)
    if name == "complete_200":
        assert want == 200 * 199 * 198 // 6  # C(n, 3)
    lib = _lib.load()
    with tc.Graph.build(s, d, n) as g:
        info = g.info()
        assert info["tasks"] <= _lib.TC_COUNT_STATIC_MAX_TASKS, name
        if name == "complete_200":
            assert 0 < info["tasks_small"] < info["tasks"]  # small and big owners both present
        assert g.count() == want
        out = torch.full((1,), -1, dtype=torch.int64, device="cuda")
        stream = torch.cuda.Stream()
        first = _static_count(lib, g, out, stream)
        out.fill_(-1)
        second = _static_count(lib, g, out, stream)
        g.check(stream)
        assert first == want and second == want, (name, first, second, want)


def test_refuses_more_tasks_than_the_array_holds():
    n = 300000
    s, d = graphgen.erdos_renyi(n, 900_000, 33)
    lib = _lib.load()
    with tc.Graph.build(s, d, n) as g:
        assert g.info()["tasks"] > _lib.TC_COUNT_STATIC_MAX_TASKS
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        rc = lib.tc_count_static(g.handle, None, ctypes.c_void_p(out.data_ptr()))
        assert rc == _lib.TC_ERR_UNSUPPORTED


def test_refuses_per_vertex_cost_models_and_null_output():
    n, s, d = F.complete(30)
    lib = _lib.load()
    with tc.Graph.build(s, d, n, tc.default_options(cost_model=tc.TC_COST_DEGREE)) as g:
        out = torch.zeros(1, dtype=torch.int64, device="cuda")
        assert lib.tc_count_static(g.handle, None, ctypes.c_void_p(out.data_ptr())) == _lib.TC_ERR_INVALID_ARG
        assert lib.tc_count_static(g.handle, None, None) == _lib.TC_ERR_INVALID_ARG


def test_takes_no_memory_from_the_graph_allocator():
    """A graph built through counting allocator hooks: the static count calls neither hook."""
    n = 50000
    s, d = graphgen.chung_lu(n, 2.2, 6.0, 800.0, 150_000, 34)
    calls = {"alloc": 0, "release": 0}
    live = {}

    @_lib.ALLOC_FN
    def alloc(ctx, nbytes, stream):
        calls["alloc"] += 1
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @_lib.RELEASE_FN
    def release(ctx, p, stream):
        calls["release"] += 1
        live.pop(p, None)

    lib = _lib.load()
    g = tc.Graph.build(s, d, n, tc.default_options(alloc=alloc, release=release))
    before = dict(calls)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    got = [_static_count(lib, g, out, stream) for _ in range(2)]
    assert calls == before
    assert got[0] == got[1] == g.count()
    g.free()
