"""Serving with continuous batching vs counts alone, through the C ABI.

Every request's total must equal the oracle's count of that graph and the library's
count of it alone (tolerance 0), however it was admitted: alone or grouped with others,
on any slot, under any budget.  The device memory in flight stays within the budget.
"""
import time

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


def _pool():
    gs = []
    for j in range(10):
        sp = W.serve_spec(j, seed=77, n_lo=2000, n_hi=60000, d_lo=8, d_hi=40)
        s, d = sp.edges()
        gs.append((s, d, sp.n))
    for j in range(6):
        sp = W.batch_spec(j, seed=78, n_lo=300, n_hi=5000, d_lo=4, d_hi=30)
        s, d = sp.edges()
        gs.append((s, d, sp.n))
    n, s, d = F.wheel(700)
    gs.append((s, d, n))
    gs.append((np.zeros(0, np.int32), np.zeros(0, np.int32), 9))
    n = 2500
    s, d = graphgen.chung_lu(n, 2.05, 150.0, 2000.0, 200_000, 79)   # lists longer than a piece
    gs.append((s, d, n))
    return gs


POOL = _pool()


@pytest.fixture(scope="module")
def want():
    alone = []
    for s, d, n in POOL:
        with tc.Graph.build(s, d, n) as g:
            alone.append(g.count())
    orc = [oracle.count_edges(n, s, d) for s, d, n in POOL]
    assert alone == orc
    return np.array(orc, np.uint64)


def _serve(server, order, pinned=False):
    graphs = POOL
    if pinned:
        graphs = [(torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory(), n) for s, d, n in POOL]
    ids = {}
    for j in order:
        s, d, n = graphs[j]
        ids[server.submit(s, d, n, tag=j)] = j
    server.drain(120_000)
    res = server.poll(10_000)
    assert len(res) == len(order)
    return res


@pytest.mark.parametrize("slots,group_edges", [(1, 1), (4, 1), (4, 0), (8, 300_000), (2, 1 << 30)])
def test_results_same_as_alone(want, slots, group_edges):
    order = list(range(len(POOL))) * 3
    with tc.Server(8 << 30, slots=slots, group_edges=group_edges) as sv:
        res = _serve(sv, order, pinned=True)
        st = sv.stats()
    for r in res:
        assert r["status"] == 0
        assert r["total"] == int(want[r["tag"]]), r
        assert r["t_submit"] <= r["t_start"] <= r["t_done"]
        assert r["slot"] < slots
    assert st["submitted"] == st["finished"] == len(order) and st["queued"] == 0
    assert st["bytes_in_flight"] == 0 and st["peak_bytes_in_flight"] <= 8 << 30
    if group_edges == 1:
        assert all(r["group"] == 1 for r in res) and st["grouped"] == 0


def test_groups_form_when_requests_wait(want):
    """Submitted faster than one slot drains them, small requests are counted in groups."""
    order = [j for j in range(len(POOL)) if POOL[j][0].size < 400_000] * 8
    with tc.Server(8 << 30, slots=1, group_edges=4_000_000) as sv:
        res = _serve(sv, order)
        st = sv.stats()
    assert st["grouped"] > 0 and max(r["group"] for r in res) > 1
    for r in res:
        assert r["status"] == 0 and r["total"] == int(want[r["tag"]])


def test_slots_overlap(want):
    order = list(range(len(POOL))) * 4
    with tc.Server(16 << 30, slots=4, group_edges=1) as sv:
        res = _serve(sv, order, pinned=True)
        st = sv.stats()
    assert st["peak_slots_busy"] > 1
    ev = sorted([(r["t_start"], 1) for r in res] + [(r["t_done"], -1) for r in res])
    live = peak = 0
    for _, e in ev:
        live += e
        peak = max(peak, live)
    assert peak > 1  # some requests ran at the same time
    for r in res:
        assert r["total"] == int(want[r["tag"]])


def test_budget_bounds_memory_in_flight(want):
    big = max(int(s.size) for s, _, _ in POOL)
    budget = 3 * 1024 * 1024 + 120 * big  # about one large request at a time
    order = list(range(len(POOL))) * 2
    with tc.Server(budget, slots=4, group_edges=0) as sv:
        res = _serve(sv, order)
        st = sv.stats()
    assert st["peak_bytes_in_flight"] <= budget
    for r in res:
        assert r["status"] == 0 and r["total"] == int(want[r["tag"]])


def test_request_above_budget_is_refused():
    s, d, n = POOL[0]
    with tc.Server(1 << 20, slots=1) as sv:
        with pytest.raises(tc.TcError) as e:
            sv.submit(s, d, n)
        assert e.value.code == _lib.TC_ERR_BUDGET


def test_bad_request_fails_alone_in_its_group(want):
    bad = (np.array([0, 1, 2], np.int32), np.array([1, 2, 50], np.int32), 10)  # id 50 >= n
    with tc.Server(8 << 30, slots=1, group_edges=1 << 30) as sv:
        big = max(range(len(POOL)), key=lambda j: POOL[j][0].size)
        sv.submit(*POOL[big][:2], POOL[big][2], tag="a")  # keep the slot busy so that the rest queue
        for j in (0, 1):
            sv.submit(*POOL[j][:2], POOL[j][2], tag=j)
        sv.submit(*bad[:2], bad[2], tag="bad")
        sv.submit(*POOL[2][:2], POOL[2][2], tag=2)
        sv.drain(60_000)
        res = {r["tag"]: r for r in sv.poll()}
    assert res["bad"]["status"] == _lib.TC_ERR_VERTEX_RANGE and res["bad"]["total"] == 0
    for j in (0, 1, 2):
        assert res[j]["status"] == 0 and res[j]["total"] == int(want[j])


def test_device_inputs_and_drain_timeout(want):
    dev = [(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n) for s, d, n in POOL]
    with tc.Server(8 << 30, slots=3) as sv:
        for j, (s, d, n) in enumerate(dev):
            sv.submit(s, d, n, tag=j)
        t0 = time.perf_counter()
        try:
            sv.drain(0)
        except tc.TcError as e:
            assert e.code == _lib.TC_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 5
        sv.drain(120_000)
        res = sv.poll()
    assert sorted(r["tag"] for r in res) == list(range(len(POOL)))
    for r in res:
        assert r["total"] == int(want[r["tag"]])


def test_destroy_with_requests_queued():
    sv = tc.Server(8 << 30, slots=1)
    for _ in range(20):
        s, d, n = POOL[0]
        sv.submit(s, d, n)
    sv.close()  # finishes what is in flight, drops the rest; must not hang


def test_cancelled_requests_leave_the_others_unchanged(want):
    """Requests withdrawn while queued come back as cancelled; every other result is exact."""
    big = max(range(len(POOL)), key=lambda j: POOL[j][0].size)
    with tc.Server(8 << 30, slots=1, group_edges=1) as sv:
        sv.submit(*POOL[big][:2], POOL[big][2], tag="busy")  # occupies the only slot
        for j in range(12):
            sv.submit(*POOL[j][:2], POOL[j][2], tag=j)
        withdrawn = sv.cancel(3) + sv.cancel(7) + sv.cancel("never submitted")
        sv.drain(120_000)
        res = {r["tag"]: r for r in sv.poll()}
    assert len(res) == 13
    cancelled = [j for j in (3, 7) if res[j]["status"] == _lib.TC_ERR_CANCELLED]
    assert len(cancelled) == withdrawn  # a request already admitted runs to the end
    for j in range(12):
        if j in cancelled:
            assert res[j]["total"] == 0 and res[j]["slot"] == -1
        else:
            assert res[j]["status"] == 0 and res[j]["total"] == int(want[j])
