"""Count over a non-overlapping partition (Sec. IV) on the GPU vs the oracle, through the C ABI.

tc_count_surrogate's P x P table (sender part i, receiving part j) must equal the oracle's
SurrogateCount table bit-exactly, for every cut pattern (one part, balanced parts, empty parts,
one vertex per part), every memory kind of the lists (pageable host, page-locked host, device,
device off a 16-byte boundary) and every range of receiving parts.  tc_surrogate_plan's cuts must
equal the oracle's Sec. IV-B cuts over the Sec. IV-F cost.
"""
import numpy as np
import pytest

import oracle
from graphgen import families as F

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on CPU only under -m gpu
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1406_5687_gb300 as tc  # noqa: E402
from paper_1406_5687_gb300 import _lib  # noqa: E402


def _graphs():
    import graphgen
    out = {
        "empty_n0": (0, np.zeros(0, np.int32), np.zeros(0, np.int32)),
        "no_edges": (17, np.zeros(0, np.int32), np.zeros(0, np.int32)),
        "k3": F.complete(3),
        "k60": F.complete(60),
        "wheel_1000": F.wheel(1000),
        "book_5000": F.book(5000),
        "star_matching": F.star_matching(3000),
        "tripartite": F.complete_tripartite(3, 40, 70),
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
    # dense: lists of up to ~800 entries (several staged pieces), runs of more than 256 entries
    # inside one part (several work items per message)
    out["dense_1400"] = F.random_graph(1400, 0.6, 7)
    return out


GRAPHS = _graphs()
CSR = {name: oracle.oriented_csr(oracle.simple_graph(n, s, d)) for name, (n, s, d) in GRAPHS.items()}


def _cut_patterns(n, seed):
    rng = np.random.default_rng(seed)
    pats = [[0, n]]
    if n >= 2:
        pats.append([0, n // 2, n])
    inner = np.sort(rng.integers(0, n + 1, 6))
    pats.append([0, 0] + inner.tolist() + [n, n])  # empty parts, first and last included
    if 0 < n <= 60:
        pats.append(list(range(n + 1)))  # one vertex per part
    elif n > 60:
        pats.append(np.linspace(0, n, 41).astype(int).tolist())
    return pats


def _expected(name, cuts):
    return oracle.count_parts(CSR[name], cuts).astype(np.uint64)


@pytest.mark.parametrize("name", [k for k in GRAPHS if k != "dense_1400"])
def test_table_matches_oracle_pageable_host(name):
    csr = CSR[name]
    T = oracle.count(csr)
    for k, cuts in enumerate(_cut_patterns(csr.n, 5)):
        total, tab = tc.count_surrogate(csr.off, csr.cols, cuts)
        exp = _expected(name, cuts)
        assert np.array_equal(tab, exp), (name, cuts)
        assert total == T


@pytest.mark.parametrize("kind", ["pinned", "device", "device_unaligned"])
@pytest.mark.parametrize("name", ["er_20k", "cl_200k", "wheel_1000", "dense_1400"])
def test_table_matches_oracle_memory_kinds(name, kind):
    csr = CSR[name]
    cuts = oracle.balanced_cuts(oracle.vertex_cost(csr, oracle.COST_NEW), 3)
    off_t = torch.from_numpy(csr.off.copy())
    cols_t = torch.from_numpy(csr.cols.copy())
    if kind == "pinned":
        off_t, cols_t = off_t.pin_memory(), cols_t.pin_memory()
    elif kind == "device":
        off_t, cols_t = off_t.cuda(), cols_t.cuda()
    else:  # device lists starting 4 bytes past a 16-byte boundary: parts are copied, not read in place
        buf = torch.empty(len(csr.cols) + 1, dtype=torch.int32, device="cuda")
        buf[1:] = cols_t.cuda()
        off_t, cols_t = off_t.cuda(), buf[1:]
        assert cols_t.data_ptr() % 16 != 0
    total, tab = tc.count_surrogate(off_t, cols_t, cuts)
    assert np.array_equal(tab, _expected(name, cuts))
    assert total == oracle.count(csr)


@pytest.mark.parametrize("name", ["ba_30k", "dense_1400"])
def test_part_ranges_add_up(name):
    """Receiving parts counted in separate calls (as on several GPUs) give the table's columns."""
    csr = CSR[name]
    n = csr.n
    cuts = [0, n // 5, n // 5, 2 * n // 5, 3 * n // 4, n]
    exp = _expected(name, cuts)
    P = len(cuts) - 1
    acc = np.zeros((P, P), np.uint64)
    for lo, hi in ((0, 2), (2, 3), (3, 5)):
        tot, tab = tc.count_surrogate(csr.off, csr.cols, cuts, part_lo=lo, part_hi=hi)
        assert np.all(tab[:, :lo] == 0) and np.all(tab[:, hi:] == 0)
        assert np.array_equal(tab[:, lo:hi], exp[:, lo:hi])
        assert tot == int(exp[:, lo:hi].sum())
        acc += tab
    assert np.array_equal(acc, exp)
    assert tc.count_surrogate(csr.off, csr.cols, cuts, part_lo=4, part_hi=4)[0] == 0


def test_dense_lists_exercise_pieces_and_split_items():
    csr = CSR["dense_1400"]
    assert csr.dhat.max() > 2 * _lib.TC_SURROGATE_PIECE  # three staged pieces
    cuts = [0, 700, 1400]
    runs = [np.count_nonzero((csr.cols[csr.off[v]:csr.off[v + 1]] >= 700)) for v in range(csr.n)]
    assert max(runs) > 256  # one message split into several work items
    total, tab = tc.count_surrogate(torch.from_numpy(csr.off).cuda(), torch.from_numpy(csr.cols).cuda(), cuts)
    assert np.array_equal(tab, _expected("dense_1400", cuts))


def test_built_graph_end_to_end():
    """tc_build's own lists, read in place on the device, counted by parts: the in-core total."""
    import graphgen
    n = 300000
    s, d = graphgen.chung_lu(n, 2.1, 24.0, 12000.0, 3_600_000, 31)
    with tc.Graph.build(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n) as g:
        T = g.count()
        _, off, cols, _ = g.csr()
        for P in (1, 4, 64):
            cuts = tc.surrogate_plan(off, cols, nparts=P)
            assert len(cuts) == P + 1
            total, tab = tc.count_surrogate(off, cols, cuts)
            assert total == T
        host_cols = cols.cpu().pin_memory()
        # parts of at most a quarter of the lists each (equal list entries, a little over 4 parts)
        cuts = tc.surrogate_plan(off, host_cols, part_bytes=host_cols.numel(), fn=tc.TC_FN_LIST)
        o = off.cpu().numpy()
        assert 4 <= len(cuts) - 1 <= 6
        assert 4 * int(np.max(o[cuts[1:]] - o[cuts[:-1]])) <= host_cols.numel()
        assert tc.count_surrogate(off.cpu(), host_cols, cuts)[0] == T


FNS = {"one": (tc.TC_FN_ONE, oracle.COST_ONE), "degree": (tc.TC_FN_DEGREE, oracle.COST_DEGREE),
       "patric": (tc.TC_FN_PATRIC, oracle.COST_PATRIC), "new": (tc.TC_FN_NEW, oracle.COST_NEW),
       "list": (tc.TC_FN_LIST, None)}


def _cost(csr, ofn):
    # TC_FN_LIST is |N_v|: the list lengths themselves
    return np.diff(csr.off).astype(np.uint64) if ofn is None else oracle.vertex_cost(csr, ofn)


@pytest.mark.parametrize("fn", list(FNS))
@pytest.mark.parametrize("name", ["er_20k", "cl_200k", "star_matching", "dense_1400", "no_edges"])
def test_plan_matches_oracle_cuts(name, fn):
    csr = CSR[name]
    gfn, ofn = FNS[fn]
    f = _cost(csr, ofn)
    for P in (1, 2, 5, 33):
        got = tc.surrogate_plan(csr.off, csr.cols, nparts=P, fn=gfn)
        assert np.array_equal(got, oracle.balanced_cuts(f, P)), (name, P)
    if csr.m_hat and fn in ("new", "list"):
        # the smallest P (from 4 m / part_bytes up to max_parts) whose balanced parts each fit;
        # on the Chung-Lu graph no P within the bound fits the equal-work cuts of Sec. IV-F
        budget = max(4 * int(csr.dhat.max()), 4 * csr.m_hat // 6)
        fit = []
        for Q in range(max(1, -(-4 * csr.m_hat // budget)), 201):
            c = oracle.balanced_cuts(f, Q)
            if 4 * int(np.max(csr.off[c[1:]] - csr.off[c[:-1]])) <= budget:
                fit = [Q]
                break
        if fit:
            got = tc.surrogate_plan(csr.off, csr.cols, part_bytes=budget, max_parts=200, fn=gfn)
            assert np.array_equal(got, oracle.balanced_cuts(f, fit[0]))
        else:
            with pytest.raises(_lib.TcError) as e:
                tc.surrogate_plan(csr.off, csr.cols, part_bytes=budget, max_parts=200, fn=gfn)
            assert e.value.code == _lib.TC_ERR_BUDGET


@pytest.mark.parametrize("name", ["er_20k", "cl_200k", "star_matching", "dense_1400"])
@pytest.mark.parametrize("work_parts", [1, 3, 5, 17])
def test_plan_both_is_the_union_of_oracle_cuts(name, work_parts):
    """Cuts bounded in work and in size: the union of the oracle's equal-work cuts (Sec. IV-F
    cost) and of its fewest equal-size cuts within the byte bound; every part then satisfies both
    bounds, and the partition still counts every triangle once."""
    csr = CSR[name]
    budget = max(4 * int(csr.dhat.max()), 4 * csr.m_hat // 4)
    fw = oracle.vertex_cost(csr, oracle.COST_NEW)
    fl = np.diff(csr.off).astype(np.uint64)
    cw = oracle.balanced_cuts(fw, work_parts)
    cb = None
    for Q in range(max(1, -(-4 * csr.m_hat // budget)), 201):
        c = oracle.balanced_cuts(fl, Q)
        if 4 * int(np.max(csr.off[c[1:]] - csr.off[c[:-1]])) <= budget:
            cb = c
            break
    assert cb is not None
    want = np.unique(np.concatenate([cw, cb]))
    got = tc.surrogate_plan_both(csr.off, csr.cols, work_parts, budget, max_parts=200)
    assert np.array_equal(got, want)
    wp = np.concatenate([[0], np.cumsum(fw.astype(np.int64))])
    work = wp[got[1:]] - wp[got[:-1]]
    assert int(work.max()) <= -(-int(wp[-1]) // work_parts) + int(fw.max())
    assert 4 * int(np.max(csr.off[got[1:]] - csr.off[got[:-1]])) <= budget
    T, _ = tc.count_surrogate(csr.off, csr.cols, got)
    assert T == oracle.count(csr)


def test_plan_budget_too_small():
    csr = CSR["wheel_1000"]
    with pytest.raises(_lib.TcError) as e:
        tc.surrogate_plan(csr.off, csr.cols, part_bytes=4 * int(csr.dhat.max()) - 4, max_parts=64,
                          fn=tc.TC_FN_LIST)
    assert e.value.code == _lib.TC_ERR_BUDGET
    with pytest.raises(_lib.TcError) as e:
        tc.surrogate_plan(csr.off, csr.cols, nparts=2, part_bytes=8)
    assert e.value.code == _lib.TC_ERR_BUDGET


def test_bad_lists_are_reported():
    """Malformed input gives a status, never a wrong count or an out-of-range access."""
    csr = CSR["er_20k"]
    n, off, cols = csr.n, csr.off, csr.cols
    cuts = [0, n // 3, n]

    def code(o, c, m=None):
        with pytest.raises(_lib.TcError) as e:
            tc.count_surrogate(o, c, cuts) if m is None else tc.surrogate_plan(o, c, nparts=2)
        return e.value.code

    v = int(np.argmax(np.diff(off) >= 3))
    a = int(off[v])
    unsorted = cols.copy()
    unsorted[a], unsorted[a + 1] = unsorted[a + 1], unsorted[a]
    assert code(off, unsorted) == _lib.TC_ERR_INVALID_ARG
    high = cols.copy()
    high[a + 2] = n + 5  # beyond every part: left unsent after the last one
    assert code(off, high) in (_lib.TC_ERR_VERTEX_RANGE, _lib.TC_ERR_INVALID_ARG)
    neg = cols.copy()
    neg[a] = -3
    assert code(off, neg) == _lib.TC_ERR_VERTEX_RANGE
    assert code(off, neg, m="plan") == _lib.TC_ERR_VERTEX_RANGE
    bad_off = off.copy()
    bad_off[5] = bad_off[6] + 1  # decreasing
    assert code(bad_off, cols) == _lib.TC_ERR_INVALID_ARG
    short = off.copy()
    short[-1] -= 1  # off[n] != number of entries
    assert code(short, cols) == _lib.TC_ERR_INVALID_ARG
    # the device stays usable, and the good lists still count right
    assert tc.count_surrogate(off, cols, cuts)[0] == oracle.count(csr)


def test_budget_and_allocator_hooks():
    csr = CSR["cl_200k"]
    cuts = oracle.balanced_cuts(oracle.vertex_cost(csr, oracle.COST_NEW), 4)
    with pytest.raises(_lib.TcError) as e:
        tc.count_surrogate(csr.off, csr.cols, cuts, options=tc.default_options(hbm_budget_bytes=1 << 16))
    assert e.value.code == _lib.TC_ERR_BUDGET
    total, tab = tc.count_surrogate(csr.off, csr.cols, cuts, options=tc.default_options(hbm_budget_bytes=1 << 30))
    assert np.array_equal(tab, _expected("cl_200k", cuts))


def test_concurrent_calls_on_the_same_pageable_lists():
    """Threads counting the same pageable host lists at once, each on its own stream: the lists
    stay page-locked until the last call ends, and every call gets the oracle's table."""
    import threading
    csr = CSR["cl_200k"]
    cuts = oracle.balanced_cuts(np.diff(csr.off).astype(np.uint64), 3)
    exp = _expected("cl_200k", cuts)
    ok, errors = [], []

    def worker():
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            for _ in range(3):
                _, tab = tc.count_surrogate(csr.off, csr.cols, cuts, stream=st)
                ok.append(np.array_equal(tab, exp))
        except Exception as e:  # reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=worker) for _ in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    assert ok == [True] * 12


def _expected_stats(csr, cuts):
    """The work tc_count_surrogate reports, from its definition on the oracle's lists: an item is a
    run of at most 256 entries of one message in one part; each item stages its whole message; each
    receiver entry u streams N_u once per staged piece of TC_SURROGATE_PIECE message entries, trimmed
    to the piece's [first, last] range when N_u has at least TC_TRIM_MIN_ENTRIES (16) entries."""
    off, cols = csr.off, csr.cols
    items = staged = streamed = 0
    for j in range(len(cuts) - 1):
        for v in range(csr.n):
            X = cols[off[v]:off[v + 1]]
            run = X[(X >= cuts[j]) & (X < cuts[j + 1])]
            if not len(run):
                continue
            d = len(X)
            k = -(-len(run) // 256)
            items += k
            staged += d * k
            L = _lib.TC_SURROGATE_PIECE
            pieces = [(p, min(p + L, d)) for p in range(0, d, L)]
            for u in run:
                Nu = cols[off[u]:off[u + 1]]
                for a, b in pieces:
                    if len(Nu) >= _lib.TC_TRIM_MIN_ENTRIES:
                        streamed += int(np.count_nonzero((Nu >= X[a]) & (Nu <= X[b - 1])))
                    else:
                        streamed += len(Nu)
    return items, staged, streamed


def test_work_counters():
    small_dense = F.random_graph(700, 0.9, 3)  # lists up to ~630 entries: three pieces
    for name, (n, s, d) in (("er_20k", GRAPHS["er_20k"]), ("small_dense", small_dense)):
        csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
        cuts = [0, n // 3, n // 2, n]
        total, tab, st = tc.count_surrogate(csr.off, csr.cols, cuts, stats=True)
        assert total == oracle.count(csr)
        items, staged, streamed = _expected_stats(csr, cuts)
        assert (st["items"], st["staged"], st["streamed"]) == (items, staged, streamed), name
        assert st["copied_bytes"] == 4 * sum(int(csr.off[b]) - (int(csr.off[a]) & ~3)
                                             for a, b in zip(cuts[:-1], cuts[1:]))
        assert st["route_ms"] > 0 and st["count_ms"] > 0
