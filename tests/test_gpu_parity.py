"""GPU path vs the CPU oracle, element by element, through the C ABI.

Integer results must match bit-exactly (tolerance 0): N+ lists and degrees (steps
a1-a5), per-edge counts (a7), totals and T_v (a8) against the oracle; the chunk
table (a6) against the oracle's Eq. 1 / Eq. 2 schedule.  The task array and the
task costs are this library's own decomposition: they are checked against its
restatement in tests/schedule_model.py, not against the oracle.
"""
import numpy as np
import pytest

import oracle
from graphgen import families as F
from graphgen import workloads as W
from tests import schedule_model as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU only under -m gpu
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1406_5687_gb300 as tc  # noqa: E402


def _graphs():
    import graphgen
    out = {
        "empty_n0": (0, np.zeros(0, np.int32), np.zeros(0, np.int32)),
        "no_edges": (17, np.zeros(0, np.int32), np.zeros(0, np.int32)),
        "k3": F.complete(3),
        "k60": F.complete(60),
        "wheel_1000": F.wheel(1000),
        "book_5000": F.book(5000),
        "tripartite": F.complete_tripartite(3, 40, 70),
        "star_matching": F.star_matching(3000),
        "friendship": F.friendship(700),
        "bipartite": F.complete_bipartite(30, 90),
        "tree": F.random_tree(5000, 1),
    }
    n = 20000
    s, d = graphgen.erdos_renyi(n, 150000, 21)
    out["er_20k"] = (n, s, d)
    n = 30000
    s, d = graphgen.barabasi_albert(n, 12, 22)
    out["ba_30k"] = (n, s, d)
    n = 200000
    s, d = graphgen.chung_lu(n, 2.1, 20.0, 8000.0, 2_000_000, 23)
    out["cl_200k"] = (n, s, d)
    n = 3000
    s, d = graphgen.chung_lu(n, 2.05, 150.0, 2500.0, 400_000, 24)  # dense: lists longer than one piece
    out["cl_dense"] = (n, s, d)
    return out


GRAPHS = _graphs()


def oracle_csr(n, s, d):
    return oracle.oriented_csr(oracle.simple_graph(n, s, d))


@pytest.fixture(scope="module")
def built():
    res = {}
    for name, (n, s, d) in GRAPHS.items():
        res[name] = (tc.Graph.build(s, d, n), oracle_csr(n, s, d))
    yield res
    for g, _ in res.values():
        g.free()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_csr_matches_oracle(built, name):
    g, csr = built[name]
    deg, off, cols, tasks = g.csr()
    assert np.array_equal(deg.cpu().numpy(), csr.deg)
    assert np.array_equal(off.cpu().numpy(), csr.off)
    assert np.array_equal(cols.cpu().numpy(), csr.cols)
    info = g.info()
    n, s, d = GRAPHS[name]
    sg = oracle.simple_graph(n, s, d)
    assert info["m_hat"] == sg.m_hat
    assert info["self_loops"] == sg.self_loops
    assert info["duplicates"] == sg.duplicates
    assert info["max_degree"] == (int(csr.deg.max()) if n else 0)
    assert info["max_dhat"] == (int(np.diff(csr.off).max()) if n else 0)
    dh = np.diff(csr.off)
    assert info["sum_dhat_v"] == int(np.repeat(dh, dh).sum())
    assert info["sum_dhat_u"] == int(dh[csr.cols].sum())


SMALL_MAX = 64  # the default build option


@pytest.mark.parametrize("name", list(GRAPHS))
def test_tasks_match_the_decomposition(built, name):
    g, csr = built[name]
    _, _, _, tasks = g.csr()
    t = tasks.cpu().numpy().astype(np.int64)
    o, p, ns = M.tasks(csr, small_max=SMALL_MAX, with_split=True)
    assert g.info()["tasks_small"] == ns
    assert np.array_equal(t[:, 0], o) and np.array_equal(t[:, 1], p)
    assert np.array_equal(t[:, 2], csr.off[p]) and np.array_equal(t[:, 3], np.diff(csr.off)[p])


@pytest.mark.parametrize("small_max", [0, 16, 256])
def test_small_max_build_option(small_max):
    for name in ("cl_200k", "cl_dense", "wheel_1000"):
        n, s, d = GRAPHS[name]
        csr = oracle_csr(n, s, d)
        with tc.Graph.build(s, d, n, tc.default_options(small_max=small_max)) as g:
            _, _, _, tasks = g.csr()
            t = tasks.cpu().numpy().astype(np.int64)
            o, p, ns = M.tasks(csr, small_max=small_max, with_split=True)
            assert g.info()["tasks_small"] == ns
            assert np.array_equal(t[:, 0], o) and np.array_equal(t[:, 1], p)
            assert g.count() == oracle.count(csr)


@pytest.mark.parametrize("name", list(GRAPHS))
def test_count_matches_oracle(built, name):
    g, csr = built[name]
    assert g.count() == oracle.count(csr)


@pytest.mark.parametrize("name", ["k60", "wheel_1000", "book_5000", "er_20k", "ba_30k", "cl_200k", "cl_dense"])
def test_per_vertex_and_per_edge(built, name):
    g, csr = built[name]
    T, pe, tv = oracle.count(csr, per_edge=True, per_vertex=True)
    T1, tv_g = g.count_per_vertex()
    assert T1 == T
    assert np.array_equal(tv_g.cpu().numpy().astype(np.uint64), tv)
    T2, pe_g = g.count_per_edge()
    assert T2 == T
    assert np.array_equal(pe_g.cpu().numpy().astype(np.uint32), pe)
    cc = g.clustering(tv_g).cpu().numpy()
    degf = csr.deg.astype(np.float64)
    want = np.where(csr.deg >= 2, 2.0 * tv.astype(np.float64) / np.maximum(degf * (degf - 1.0), 1.0), 0.0)
    assert np.array_equal(cc, want)


def _hub_fan(k, L):
    """A clique on {0} + W (W = 1..k), L leaves each adjacent to 0 and 1, and pendants that
    lift every vertex of W above vertex 0 in the degree order (deg 0 = k + L)."""
    iu = np.triu_indices(k + 1, 1)
    s = [iu[0], np.arange(k + 1, k + 1 + L), np.arange(k + 1, k + 1 + L)]
    d = [iu[1], np.zeros(L, np.int64), np.ones(L, np.int64)]
    nxt = k + 1 + L
    for w, extra in [(1, 1)] + [(j, L + 1) for j in range(2, k + 1)]:
        s.append(np.full(extra, w, np.int64))
        d.append(np.arange(nxt, nxt + extra))
        nxt += extra
    return nxt, np.concatenate(s).astype(np.int32), np.concatenate(d).astype(np.int32)


@pytest.mark.parametrize("k,piece", [(3, 2048), (257, 256)])
def test_per_vertex_many_hits_at_one_slot(k, piece):
    """Vertex 0 owns all the L = 70,000 leaf tasks (its list W is longer than a leaf's {0, 1}),
    each finding the triangle (0, leaf, 1) at vertex 1's slot of 0's table: 70,000 hits at one
    slot (more than 16 bits hold), all in one chunk (every owner big, no static share, one
    guided chunk).  k = 3 stages 0's list in a window of owners; k = 257 with pieces of 256
    entries stages it in two pieces.  Closed forms: T = C(k+1, 3) + L; T_0 = T_1 = C(k, 2) + L,
    T_w = C(k, 2) for the rest of W, 1 per leaf, 0 per pendant."""
    L = 70000
    n, s, d = _hub_fan(k, L)
    opt = tc.default_options(small_max=0, piece=piece, static_percent=0, min_chunk=1 << 60)
    ck2, ck3 = k * (k - 1) // 2, (k + 1) * k * (k - 1) // 6
    with tc.Graph.build(s, d, n, opt) as g:
        assert g.info()["tasks"] > g.info()["tasks_small"]
        T, tv = g.count_per_vertex()
        assert T == ck3 + L
        tv = tv.cpu().numpy()
        assert tv[0] == ck2 + L and tv[1] == ck2 + L
        assert (tv[2:k + 1] == ck2).all()
        assert (tv[k + 1:k + 1 + L] == 1).all()
        assert not tv[k + 1 + L:].any()
        T2, pe = g.count_per_edge()
        assert T2 == T and int(pe.sum().item()) == T


@pytest.mark.parametrize("name", ["wheel_1000", "er_20k", "cl_200k", "cl_dense"])
@pytest.mark.parametrize("fn", [tc.TC_FN_ONE, tc.TC_FN_DEGREE, tc.TC_FN_PATRIC, tc.TC_FN_NEW])
def test_vertex_cost(built, name, fn):
    g, csr = built[name]
    f = g.vertex_cost(fn).cpu().numpy().astype(np.uint64)
    assert np.array_equal(f, oracle.vertex_cost(csr, fn))


def _sorted_rows(x):
    return x[np.lexsort(tuple(x[:, k] for k in range(x.shape[1] - 1, -1, -1)))]


@pytest.mark.parametrize("name", ["er_20k", "cl_200k", "cl_dense", "book_5000"])
@pytest.mark.parametrize("model,piece", [(tc.TC_COST_EDGE, 2048), (tc.TC_COST_EDGE, 256), (tc.TC_COST_MERGE, 512),
                                         (tc.TC_COST_DEGREE, 1024), (tc.TC_COST_PATRIC, 2048),
                                         (tc.TC_COST_NEW, 4096), (tc.TC_COST_ONE, 2048)])
def test_schedule_matches_oracle(built, name, model, piece):
    """Per class, the chunks the workers took are exactly the oracle's Eq. 1 + Eq. 2 schedule over
    the task costs (the paper's merge and per-vertex costs, or this design's EDGE cost)."""
    g, csr = built[name]
    big_warps = 16 if piece <= 2048 else 8
    opt = tc.default_options(cost_model=model, piece=piece, warps_per_block=16, big_warps=big_warps)
    T, meta, chunks, busy = g.count_ex(opt, trace_cap=1 << 20, busy=True)
    assert T == oracle.count(csr)
    o, p, ns = M.tasks(csr, small_max=SMALL_MAX, with_split=True)
    assert meta["tasks_small"] == ns
    if model == tc.TC_COST_EDGE:
        cost = M.task_costs(csr, o, p, M.MODEL_EDGE, piece=piece, c_task=4, c_owner=32,
                                 small_max=SMALL_MAX)
    elif model == tc.TC_COST_MERGE:
        cost = M.task_costs(csr, o, p, M.MODEL_MERGE)
    else:
        cost = M.task_costs(csr, o, p, M.MODEL_VERTEX, fn=model - tc.TC_COST_ONE)
    got = chunks.cpu().numpy()
    n_want = 0
    for cls, (lo, hi) in enumerate(((0, ns), (ns, len(o)))):
        c = cost[lo:hi]
        assert meta["total_cost"][cls] == int(c.sum())
        mine = got[got[:, 0] == cls][:, 1:]
        if hi == lo:
            assert len(mine) == 0  # an empty class launches no kernel
            continue
        cb, tb = oracle.schedule(c, meta["n_workers"][cls], meta["min_chunk"][cls])
        want = np.stack([cb[:-1], cb[1:], tb[:-1] + lo, tb[1:] + lo], axis=1).astype(np.int64)
        n_want += len(want)
        # static chunks are recorded per worker, dynamic ones in pop order: compare as sorted rows
        assert np.array_equal(_sorted_rows(mine), _sorted_rows(want))
    assert meta["n_chunks"] == n_want == len(got)
    b = busy.cpu().numpy()
    W = meta["n_workers"]
    assert b.shape[0] == W[0] + W[1]
    if ns > 0:
        assert int(b[:W[0], 1].sum()) == int((got[:, 0] == 0).sum())
    if len(o) > ns:
        assert int(b[W[0]:, 1].sum()) == int((got[:, 0] == 1).sum())


@pytest.mark.parametrize("static_percent", [0, 25, 50, 100])
@pytest.mark.parametrize("min_chunk", [0, 1, 100000])
def test_schedule_parameters_keep_the_count(built, static_percent, min_chunk):
    g, csr = built["cl_200k"]
    opt = tc.default_options(static_percent=static_percent, min_chunk=min_chunk)
    T, *_ = g.count_ex(opt)
    assert T == oracle.count(csr)


@pytest.mark.parametrize("wpb,piece,bps,bw", [(1, 256, 0, 4), (4, 512, 2, 8), (16, 1024, 1, 16), (4, 2048, 0, 16),
                                           (8, 4096, 1, 8), (2, 256, 3, 16)])
def test_launch_shapes_keep_the_count(built, wpb, piece, bps, bw):
    for name in ("cl_dense", "cl_200k", "ba_30k"):
        g, csr = built[name]
        opt = tc.default_options(warps_per_block=wpb, piece=piece, blocks_per_sm=bps, big_warps=bw)
        T, *_ = g.count_ex(opt)
        assert T == oracle.count(csr)


def test_device_input_and_dirty_input():
    n, s, d = GRAPHS["cl_200k"]
    rng = np.random.default_rng(5)
    pick = rng.integers(0, len(s), 5000)
    s2 = np.concatenate([s, d[pick], np.arange(100, dtype=np.int32)])
    d2 = np.concatenate([d, s[pick], np.arange(100, dtype=np.int32)])
    order = rng.permutation(len(s2))
    s2, d2 = s2[order], d2[order]
    sg = oracle.simple_graph(n, s2, d2)
    T = oracle.count(oracle.oriented_csr(sg))
    with tc.Graph.build(torch.from_numpy(s2).cuda(), torch.from_numpy(d2).cuda(), n) as g:
        info = g.info()
        assert (info["m_hat"], info["self_loops"], info["duplicates"]) == (sg.m_hat, sg.self_loops, sg.duplicates)
        assert g.count() == T


def test_input_errors():
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(np.array([0, 5], np.int32), np.array([1, 2], np.int32), 5)
    assert e.value.code == tc._lib.TC_ERR_VERTEX_RANGE
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(np.array([0, -3], np.int32), np.array([1, 2], np.int32), 5)
    assert e.value.code == tc._lib.TC_ERR_VERTEX_RANGE
    strict = tc.default_options(input_policy=tc.TC_INPUT_STRICT)
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(np.array([0, 1], np.int32), np.array([1, 0], np.int32), 5, strict)
    assert e.value.code == tc._lib.TC_ERR_INVALID_ARG
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(np.array([2], np.int32), np.array([2], np.int32), 5, strict)
    assert e.value.code == tc._lib.TC_ERR_INVALID_ARG
    with tc.Graph.build(np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32), 3, strict) as g:
        assert g.count() == 1


def test_budget_and_allocator_failure():
    n, s, d = GRAPHS["er_20k"]
    small = tc.default_options(hbm_budget_bytes=1 << 16)
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(s, d, n, small)
    assert e.value.code == tc._lib.TC_ERR_BUDGET

    calls = {"n": 0}

    @tc._lib.ALLOC_FN
    def failing_alloc(ctx, nbytes, stream):
        calls["n"] += 1
        return None

    @tc._lib.RELEASE_FN
    def release(ctx, p, stream):
        pass

    opt = tc.default_options(alloc=failing_alloc, release=release)
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(s, d, n, opt)
    assert e.value.code == tc._lib.TC_ERR_OOM and calls["n"] >= 1


def test_caller_allocator_is_used():
    """Device memory can come from torch's caching allocator through the hooks."""
    n, s, d = GRAPHS["ba_30k"]
    live = {}

    @tc._lib.ALLOC_FN
    def alloc(ctx, nbytes, stream):
        t = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        return t.data_ptr()

    @tc._lib.RELEASE_FN
    def release(ctx, p, stream):
        live.pop(p, None)

    opt = tc.default_options(alloc=alloc, release=release)
    g = tc.Graph.build(s, d, n, opt)
    assert len(live) > 0
    assert g.count() == oracle.count(oracle_csr(n, s, d))
    g.free()
    assert len(live) == 0


def test_async_count_and_graph_capture(built):
    g, csr = built["cl_200k"]
    T = oracle.count(csr)
    out = torch.zeros(1, dtype=torch.int64, device="cuda")
    g.count_async(out)
    g.check()
    assert int(out.item()) == T
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        g.count_async(out)  # warm-up on the capture stream: the workspace already exists
    s.synchronize()
    cg = torch.cuda.CUDAGraph()
    out2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    with torch.cuda.graph(cg, stream=s):
        g.count_async(out2, stream=s)
    for _ in range(3):
        out2.zero_()
        cg.replay()
        torch.cuda.synchronize()
        assert int(out2.item()) == T


def test_er_golden():
    """The ER workload's stored oracle values (tests/golden/er_10k.txt)."""
    import os
    gold = {}
    with open(os.path.join(os.path.dirname(__file__), "golden", "er_10k.txt")) as f:
        for line in f:
            if not line.startswith("#"):
                k, v = line.split()
                gold[k] = v
    s, d = W.ER_10K.edges()
    with tc.Graph.build(s, d, W.ER_10K.n) as g:
        assert g.info()["m_hat"] == int(gold["m_hat"])
        assert g.count() == int(gold["triangles"])
        T, tv = g.count_per_vertex()
        assert int(tv.sum().item()) == int(gold["sum_t_v"])


def test_bounded_wait_gives_up_and_the_context_survives():
    """A device wait on a flag that nothing sets returns TC_ERR_TIMEOUT after its limit."""
    from paper_1406_5687_gb300 import _lib
    lib = _lib.load()
    stream = torch.cuda.current_stream()
    for limit in (1, 1000, 100_000):
        assert lib.tc_wait_selftest(limit, tc._stream(stream)) == _lib.TC_ERR_TIMEOUT
    assert lib.tc_wait_selftest(0, None) == _lib.TC_ERR_INVALID_ARG
    n, s, d = GRAPHS["cl_200k"]
    with tc.Graph.build(s, d, n) as g:
        assert g.count() == oracle.count(oracle_csr(n, s, d))


def test_tiny_wait_limits_fail_cleanly_or_count_exactly():
    """With a look-back / queue limit of a few polls a build or count may give up: it then
    reports TC_ERR_TIMEOUT instead of a wrong total, and the next call works."""
    n, s, d = GRAPHS["cl_200k"]
    want = oracle.count(oracle_csr(n, s, d))
    for limit in (1, 4):
        try:
            with tc.Graph.build(s, d, n, tc.default_options(retry_limit=limit)) as g:
                assert g.count() == want
        except tc.TcError as e:
            assert e.code == tc._lib.TC_ERR_TIMEOUT
    with tc.Graph.build(s, d, n) as g:
        assert g.count() == want


def _streamed_entries(csr, small_max, piece, trim_min=None):
    """Partner entries each class's kernel must read: a small owner's partner list whole;
    for a big owner, per piece of its list (pieces of `piece` entries), the part of the
    partner list within the piece's [first, last] entries (both lists are ascending) when the
    partner list has at least trim_min entries, else the whole list."""
    from paper_1406_5687_gb300 import _lib
    trim_min = _lib.TC_TRIM_MIN_ENTRIES if trim_min is None else trim_min
    own, par, ns = M.tasks(csr, small_max=small_max, with_split=True)
    off, cols = csr.off, csr.cols.astype(np.int64)
    dh = np.diff(off)
    small = int(dh[par[:ns]].sum())
    o, p = own[ns:].astype(np.int64), par[ns:].astype(np.int64)
    key = cols + np.repeat(np.arange(len(dh), dtype=np.int64), dh) * (1 << 32)
    big = 0
    npieces = (dh[o] + piece - 1) // piece
    for k in range(int(npieces.max()) if len(o) else 0):
        m = npieces > k
        ob = off[o[m]] + k * piece
        pl = np.minimum(piece, dh[o[m]] - k * piece)
        lo_v, hi_v = cols[ob], cols[ob + pl - 1]
        pm = p[m]
        lo = np.searchsorted(key, pm * (1 << 32) + lo_v, side="left")
        hi = np.searchsorted(key, pm * (1 << 32) + hi_v, side="right")
        whole = dh[pm] < trim_min
        big += int(np.where(whole, dh[pm], hi - lo).sum())
    return small, big


@pytest.mark.parametrize("name,piece", [("cl_200k", 2048), ("cl_dense", 256), ("ba_30k", 1024)])
def test_streamed_entries_match_the_host_count(name, piece):
    n, s, d = GRAPHS[name]
    csr = oracle_csr(n, s, d)
    want = _streamed_entries(csr, 64, piece)
    with tc.Graph.build(s, d, n) as g:
        T, meta, _, _ = g.count_ex(tc.default_options(piece=piece), streamed=True)
        assert T == oracle.count(csr)
        assert tuple(meta["streamed"]) == want
        _, meta2, _, _ = g.count_ex(tc.default_options(piece=piece), timing=True)
        assert list(meta2["streamed"]) == [-1, -1]


@pytest.mark.parametrize("shift", [0, 1, 2, 3, 4])
def test_unaligned_and_ragged_device_edge_lists(shift):
    """Edge lists that start off a 16-byte boundary, or whose length is not a multiple of 4,
    take the canonicalize kernel's scalar path; the count is the same."""
    n, s, d = GRAPHS["ba_30k"]
    want = oracle.count(oracle_csr(n, s[shift:len(s) - shift], d[shift:len(d) - shift]))
    sd, dd = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    with tc.Graph.build(sd[shift:len(s) - shift], dd[shift:len(d) - shift], n) as g:
        assert g.count() == want
    bad = dd.clone()
    bad[len(d) - 1 - shift] = n  # an out-of-range id in the ragged tail
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(sd[shift:len(s) - shift], bad[shift:len(d) - shift], n)
    assert e.value.code == tc._lib.TC_ERR_VERTEX_RANGE


@pytest.mark.parametrize("m", [8191, 8192, 8193, 3 * 8192 + 1, 4096 * 3 - 1])
def test_sort_tile_boundaries(m):
    """Edge lists of about one, two and three radix-sort tiles (8192 keys each), on either side of
    a tile's end, with repeats, self-loops and hubs: the lists, degrees and count equal the
    oracle's (bit-exact)."""
    rng = np.random.default_rng(m)
    n = 3000
    hub = rng.integers(0, 20, size=m)                    # a few hubs take most edges
    other = rng.integers(0, n, size=m)
    pick = rng.random(m) < 0.5
    s = np.where(pick, hub, other).astype(np.int32)
    d = rng.integers(0, n, size=m).astype(np.int32)
    d[::97] = s[::97]                                    # self-loops
    s[1::53], d[1::53] = s[0:-1:53][: len(s[1::53])], d[0:-1:53][: len(d[1::53])]  # repeats
    csr = oracle_csr(n, s, d)
    with tc.Graph.build(s, d, n) as g:
        deg, off, cols, _ = g.csr()
        assert np.array_equal(deg.cpu().numpy(), csr.deg)
        assert np.array_equal(off.cpu().numpy(), csr.off)
        assert np.array_equal(cols.cpu().numpy(), csr.cols)
        assert g.count() == oracle.count(csr)


@pytest.mark.parametrize("name", ["cl_200k", "cl_dense", "ba_30k", "k60", "no_edges"])
@pytest.mark.parametrize("nparts", [1, 2, 3, 7, 64])
def test_partitioned_count_adds_up(name, nparts):
    """Cost-balanced parts of the tasks (Sec. IV-B's partition of the a6 costs) cover every
    task once: the partial counts sum to T."""
    n, s, d = GRAPHS[name]
    want = oracle.count(oracle_csr(n, s, d))
    with tc.Graph.build(s, d, n) as g:
        parts = [g.count_partition(p, nparts) for p in range(nparts)]
        assert sum(parts) == want, parts
        assert g.count() == want  # the full count is unaffected


def _part_counts(csr, nparts, model, piece=2048, small_max=SMALL_MAX):
    """Per part, the oracle's per-edge counts (Theorem 1 attribution) summed over the oriented
    edges of the tasks that part holds: per class, the tasks whose exclusive cost prefix lies in
    [C p / P, C (p + 1) / P)."""
    _, pe, _ = oracle.count(csr, per_edge=True, per_vertex=True)
    o, p, ns, pos = M.tasks(csr, small_max=small_max, with_split=True, with_pos=True)
    if model == tc.TC_COST_EDGE:
        cost = M.task_costs(csr, o, p, M.MODEL_EDGE, piece=piece, c_task=4, c_owner=32, small_max=small_max)
    elif model == tc.TC_COST_MERGE:
        cost = M.task_costs(csr, o, p, M.MODEL_MERGE)
    else:
        cost = M.task_costs(csr, o, p, M.MODEL_VERTEX, fn=model - tc.TC_COST_ONE)
    want = np.zeros(nparts, np.int64)
    for lo, hi in ((0, ns), (ns, len(o))):
        part = M.partition_members(cost[lo:hi], nparts)
        np.add.at(want, part, pe[pos[lo:hi]].astype(np.int64))
    return want


@pytest.mark.parametrize("name", ["cl_200k", "cl_dense", "ba_30k", "book_5000"])
@pytest.mark.parametrize("nparts", [2, 3, 7, 64])
@pytest.mark.parametrize("model", [tc.TC_COST_EDGE, tc.TC_COST_MERGE, tc.TC_COST_DEGREE, tc.TC_COST_NEW])
def test_each_partition_part_counts_its_own_tasks(name, nparts, model):
    """Every part, not only their sum: part p's count equals the oracle's per-edge counts of
    exactly the oriented edges whose tasks fall in part p, so no part counts a task twice
    while another misses it."""
    n, s, d = GRAPHS[name]
    csr = oracle_csr(n, s, d)
    want = _part_counts(csr, nparts, model)
    with tc.Graph.build(s, d, n, tc.default_options(cost_model=model)) as g:
        got = [g.count_partition(p, nparts) for p in range(nparts)]
    assert got == want.tolist()
    assert int(want.sum()) == oracle.count(csr)


@pytest.mark.parametrize("options", [dict(cost_model=tc.TC_COST_DEGREE), dict(cost_model=tc.TC_COST_NEW),
                                     dict(static_percent=0), dict(static_percent=100)])
def test_partitioned_count_with_per_vertex_costs(options):
    """Per-vertex cost models give zero-cost tasks (an owner's cost sits on its last task), so
    parts may meet inside an owner's tasks; they still cover every task once."""
    n, s, d = GRAPHS["cl_200k"]
    want = oracle.count(oracle_csr(n, s, d))
    with tc.Graph.build(s, d, n, tc.default_options(**options)) as g:
        for nparts in (2, 5):
            assert sum(g.count_partition(p, nparts) for p in range(nparts)) == want


def test_partition_arguments():
    n, s, d = GRAPHS["k3"]
    with tc.Graph.build(s, d, n) as g:
        for part, nparts in [(0, 0), (2, 2), (-1, 3)]:
            with pytest.raises(tc.TcError) as e:
                g.count_partition(part, nparts)
            assert e.value.code == tc._lib.TC_ERR_INVALID_ARG


def test_largest_vertex_count():
    """n = 2^30, the largest supported: K_5 on the five highest ids and a wheel W_100 on the
    lowest, so T = C(5,3) + 99 by the closed forms, with per-vertex counts at both ends."""
    n = 1 << 30
    top = np.arange(n - 5, n, dtype=np.int64)
    iu = np.triu_indices(5, 1)
    s1, d1 = top[iu[0]], top[iu[1]]
    wn, ws, wd = F.wheel(100)
    s = np.concatenate([s1, ws.astype(np.int64)]).astype(np.int32)
    d = np.concatenate([d1, wd.astype(np.int64)]).astype(np.int32)
    with tc.Graph.build(s, d, n) as g:
        assert g.count() == 10 + 99
        T, tv = g.count_per_vertex()
        assert T == 109
        assert tv[n - 5:].tolist() == [6] * 5          # each K_5 vertex is in C(4,2) triangles
        assert int(tv[:100].sum().item()) == 3 * 99
        assert sum(g.count_partition(p, 3) for p in range(3)) == 109
    with pytest.raises(tc.TcError) as e:
        tc.Graph.build(s, d, n + 1)
    assert e.value.code == tc._lib.TC_ERR_UNSUPPORTED
