"""Batched counting vs the CPU oracle, graph by graph, through the C ABI.

Each graph of a batch must get exactly the oracle's total for that graph alone
(tolerance 0: counts are integers), whatever the packing, the launch shape, the
cost model or the number of replays; so must its distinct edge count.
"""
import ctypes

import numpy as np
import pytest

import oracle
from graphgen import families as F
from graphgen import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import graphgen  # noqa: E402
import paper_1406_5687_gb300 as tc  # noqa: E402
from paper_1406_5687_gb300 import _lib  # noqa: E402


def _mixed():
    """Small graphs of every kind, including empty ones and dirty input."""
    gs = []
    for j in range(24):
        sp = W.batch_spec(j, seed=97, n_lo=200, n_hi=6000, d_lo=4, d_hi=40)
        s, d = sp.edges()
        gs.append((s, d, sp.n))
    n, s, d = F.complete(40)
    gs.insert(3, (s, d, n))
    n, s, d = F.wheel(900)
    gs.insert(7, (s, d, n))
    gs.insert(0, (np.zeros(0, np.int32), np.zeros(0, np.int32), 0))        # n = 0
    gs.insert(5, (np.zeros(0, np.int32), np.zeros(0, np.int32), 50))       # no edges
    n = 3000
    s, d = graphgen.chung_lu(n, 2.05, 150.0, 2500.0, 300_000, 41)          # lists longer than a piece
    gs.append((s, d, n))
    # dirty: self-loops, repeats and reversed pairs, merged by the input policy
    n, s, d = F.complete(25)
    s2 = np.concatenate([s, d, np.arange(25, dtype=np.int32), s[:50]])
    d2 = np.concatenate([d, s, np.arange(25, dtype=np.int32), d[:50]])
    gs.append((s2, d2, n))
    return gs


MIXED = _mixed()


def _want(graphs):
    T, mh = [], []
    for s, d, n in graphs:
        csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
        T.append(oracle.count(csr))
        mh.append(csr.m_hat)
    return np.array(T, np.uint64), np.array(mh, np.int64)


@pytest.fixture(scope="module")
def want():
    return _want(MIXED)


def test_totals_and_edges_match_the_oracle(want):
    T, mh = want
    with tc.Batch.build(MIXED) as b:
        got = b.count()
        assert np.array_equal(got, T), (got, T)
        assert np.array_equal(b.graph_edges(), mh)
        info = b.info()
        assert info["k"] == len(MIXED) and info["packs"] == 1
        assert info["m_hat"] == int(mh.sum())


@pytest.mark.parametrize("pack_edges", [1, 20_000, 150_000])
def test_any_packing_gives_the_same_totals(want, pack_edges):
    T, _ = want
    with tc.Batch.build(MIXED, pack_edges=pack_edges) as b:
        info = b.info()
        if pack_edges == 1:
            assert info["packs"] == len(MIXED)  # every graph a pack of its own
        else:
            assert 1 < info["packs"] < len(MIXED)
        assert np.array_equal(b.count(), T)


def test_replays_and_device_output(want):
    T, _ = want
    with tc.Batch.build(MIXED, pack_edges=100_000) as b:
        out = torch.full((len(MIXED) + 3,), -1, dtype=torch.int64, device="cuda")
        stream = torch.cuda.Stream()
        l0 = tc.kernel_launches()
        for _ in range(3):
            b.run(out, stream)
        b.check(stream)
        assert tc.kernel_launches() > l0
        got = out.cpu().numpy()
        assert np.array_equal(got[:len(MIXED)].astype(np.uint64), T)
        assert np.all(got[len(MIXED):] == -1)  # nothing written past k


@pytest.mark.parametrize("shape", [dict(warps_per_block=4, big_warps=8, piece=1024),
                                   dict(warps_per_block=8, big_warps=16, piece=256, static_percent=0),
                                   dict(warps_per_block=16, big_warps=4, piece=4096, static_percent=100),
                                   dict(cost_model=tc.TC_COST_DEGREE), dict(cost_model=tc.TC_COST_MERGE)])
def test_launch_shapes_and_cost_models(want, shape):
    T, _ = want
    with tc.Batch.build(MIXED) as b:
        assert np.array_equal(b.count(), T)
        b.set_options(tc.default_options(**shape))
        assert np.array_equal(b.count(), T)


@pytest.mark.parametrize("small_max", [0, 16, 256])
def test_hub_thresholds(want, small_max):
    T, _ = want
    with tc.Batch.build(MIXED, options=tc.default_options(small_max=small_max)) as b:
        assert np.array_equal(b.count(), T)
        with pytest.raises(tc.TcError):  # build-time field: cannot change after the build
            b.set_options(tc.default_options(small_max=64 if small_max != 64 else 32))


def test_device_edge_lists(want):
    T, _ = want
    dev = [(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n) for s, d, n in MIXED]
    with tc.Batch.build(dev, pack_edges=50_000) as b:
        assert np.array_equal(b.count(), T)


def test_id_out_of_its_own_graph_is_an_error():
    # vertex 10 exists in the union (the next graph's range) but not in graph 1
    gs = [F.complete(12)[1:] + (12,), (np.array([0, 1], np.int32), np.array([1, 10], np.int32), 10),
          F.complete(12)[1:] + (12,)]
    with pytest.raises(tc.TcError) as e:
        tc.Batch.build(gs)
    assert e.value.code == _lib.TC_ERR_VERTEX_RANGE
    with pytest.raises(tc.TcError) as e:
        tc.Batch.build([(np.array([-1], np.int32), np.array([0], np.int32), 5)])
    assert e.value.code == _lib.TC_ERR_VERTEX_RANGE


def test_empty_batch_and_bad_arguments():
    with tc.Batch.build([]) as b:
        assert b.count().size == 0
        assert b.info()["k"] == 0
    lib = _lib.load()
    h = ctypes.c_void_p()
    m = np.array([-1], np.int64)
    n = np.array([3], np.int32)
    srcs = (ctypes.c_void_p * 1)()
    assert lib.tc_batch_build(srcs, srcs, m.ctypes.data_as(ctypes.c_void_p), n.ctypes.data_as(ctypes.c_void_p),
                              1, 0, None, None, ctypes.byref(h)) == _lib.TC_ERR_INVALID_ARG
    assert lib.tc_batch_run(None, None, None) == _lib.TC_ERR_INVALID_ARG


def test_disjoint_union_equals_the_batch(want):
    """The batch's totals add up to the count of the same graphs built as one graph."""
    T, _ = want
    parts = [(n, s, d) for s, d, n in MIXED]
    n, s, d = F.disjoint_union(*parts)
    with tc.Graph.build(s, d, n) as g:
        assert g.count() == int(T.sum())


def test_autotune_returns_a_candidate_that_counts_exactly(want):
    T, _ = want
    best, rep = tc.autotune(MIXED, reps=1)
    assert rep["tried"] == 3 * 3 * 2 * 2 and len(rep["candidates"]) == rep["tried"]
    assert rep["best_ms"] > 0 and rep["best_ms"] == min(c["ms"] for c in rep["candidates"])
    assert rep["default_ms"] > 0
    assert best.small_max in (32, 64, 128) and best.warps_per_block in (4, 8, 16)
    with tc.Batch.build(MIXED, options=best) as b:
        assert np.array_equal(b.count(), T)


def test_autotune_cache_returns_the_stored_choice(tmp_path, want):
    T, _ = want
    path = str(tmp_path / "tune.json")
    best, rep = tc.autotune(MIXED, reps=1, cache_path=path)
    assert rep["cached"] is False and rep["signature"]
    again, rep2 = tc.autotune(MIXED, reps=1, cache_path=path)
    assert rep2["cached"] is True and rep2["signature"] == rep["signature"]
    for k in ("small_max", "warps_per_block", "big_warps", "piece", "static_percent"):
        assert getattr(again, k) == getattr(best, k)
    with tc.Batch.build(MIXED, options=again) as b:
        assert np.array_equal(b.count(), T)
