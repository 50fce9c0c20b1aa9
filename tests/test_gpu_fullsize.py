"""Full-size workloads in the benchmark's launch configuration (default options).

The totals are compared with the oracle's own count of the same graph (its Fig. 1 loop
split over the host cores; the integer sum is exact in any order), and sampled
per-edge counts with intersections of the oracle's lists computed one by one.
"""
import os

import numpy as np
import pytest

import oracle
from graphgen import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_1406_5687_gb300 as tc  # noqa: E402

THREADS = os.cpu_count() or 1


@pytest.mark.parametrize("name", ["ba", "cl"])
def test_full_size_total_and_sampled_edges(name):
    spec = W.SINGLE[name]
    s, d = spec.edges()
    csr = oracle.oriented_csr(oracle.simple_graph(spec.n, s, d))
    T_oracle = oracle.count(csr, threads=THREADS)
    sd, dd = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    del s, d
    with tc.Graph.build(sd, dd, spec.n) as g:
        del sd, dd
        info = g.info()
        assert info["m_hat"] == csr.m_hat
        T = g.count()
        assert T == T_oracle
        assert g.count() == T  # repeated launches agree
        T2, pe = g.count_per_edge()
        assert T2 == T
        rng = np.random.default_rng(7)
        idx = rng.integers(0, csr.m_hat, 2000)
        rows = np.searchsorted(csr.off, idx, side="right") - 1
        pe_h = pe.cpu().numpy()
        for i, v in zip(idx.tolist(), rows.tolist()):
            u = int(csr.cols[i])
            a = csr.cols[csr.off[v]:csr.off[v + 1]]
            b = csr.cols[csr.off[u]:csr.off[u + 1]]
            assert int(pe_h[i]) == len(np.intersect1d(a, b, assume_unique=True)), (v, u)
        T3, tv = g.count_per_vertex()
        assert T3 == T and int(tv.sum().item()) == 3 * T


def _spread(specs, k):
    """k specs spread over the list (the workload's range of sizes), smallest input first."""
    step = max(1, len(specs) // k)
    return sorted(specs[::step][:k], key=lambda sp: sp.num_input_edges)


@pytest.mark.parametrize("options", [{}, dict(small_max=128, warps_per_block=16, big_warps=8, piece=2048)])
def test_batch_workload_sample(options):
    """Every 16th graph of the 4096-graph batch workload, in packs of at most 2^29 input edges
    as the bench builds them: each total equals the graph counted alone, and sampled graphs
    equal the oracle."""
    specs = W.batch_specs()[::16]
    graphs = [sp.edges() + (sp.n,) for sp in specs]
    opt = tc.default_options(**options)
    with tc.Batch.build(graphs, options=opt, pack_edges=1 << 29) as b:
        totals = b.count()
        edges = b.graph_edges()
    for j, (s, d, n) in enumerate(graphs):
        with tc.Graph.build(s, d, n, opt) as g:
            assert g.count() == int(totals[j]), j
            assert g.info()["m_hat"] == int(edges[j])
    for sp in _spread(specs, 6):
        j = specs.index(sp)
        s, d, n = graphs[j]
        assert oracle.count(oracle.oriented_csr(oracle.simple_graph(n, s, d)), threads=THREADS) == int(totals[j]), j


def test_serve_workload_sample():
    """The first 24 graphs of the serving pool, served by 4 slots with grouping: every total
    equals the graph counted alone, and the smaller ones equal the oracle."""
    specs = [W.serve_spec(j) for j in range(24)]
    graphs = [(torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory(), sp.n)
              for sp in specs for s, d in [sp.edges()]]
    with tc.Server(60 << 30, slots=4) as sv:
        for j, (s, d, n) in enumerate(graphs):
            sv.submit(s, d, n, tag=j)
        sv.drain(600_000)
        res = {r["tag"]: r for r in sv.poll(100)}
    assert sorted(res) == list(range(len(graphs)))
    for j, (s, d, n) in enumerate(graphs):
        assert res[j]["status"] == 0
        with tc.Graph.build(s, d, n) as g:
            assert g.count() == res[j]["total"], j
        if specs[j].num_input_edges <= 4_000_000:
            want = oracle.count(oracle.oriented_csr(oracle.simple_graph(n, s.numpy(), d.numpy())), threads=THREADS)
            assert want == res[j]["total"], j


@pytest.mark.slow
def test_twitter_size_chung_lu():
    """A Chung-Lu graph of the size of the paper's largest real graph (Twitter, Table I:
    41.65M vertices, 2.4e9 edge draws), built and counted in device memory.  Too large for the
    oracle's single-thread list build, so the checks are the method's own identities: the
    cost-balanced parts sum to T, sum T_v = 3T, the per-edge counts sum to T, sampled per-edge
    counts equal intersections of the built lists computed on the host, and the sampled lists
    are ascending and oriented by the order of Sec. III-A."""
    spec = W.SINGLE["cl_twitter"]
    s, d = spec.edges()
    sd, dd = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    del s, d
    with tc.Graph.build(sd, dd, spec.n) as g:
        del sd, dd
        info = g.info()
        T = g.count()
        assert sum(g.count_partition(p, 4) for p in range(4)) == T
        T2, tv = g.count_per_vertex()
        assert T2 == T and int(tv.sum().item()) == 3 * T
        del tv
        T3, pe = g.count_per_edge()
        assert T3 == T and int(pe.sum().item()) == T
        deg, off, cols, tasks = g.csr()
        del tasks
        off, cols, deg, pe = off.cpu().numpy(), cols.cpu().numpy(), deg.cpu().numpy(), pe.cpu().numpy()
    assert int(off[-1]) == info["m_hat"]
    rng = np.random.default_rng(11)
    idx = rng.integers(0, info["m_hat"], 2000)
    rows = np.searchsorted(off, idx, side="right") - 1
    for i, v in zip(idx.tolist(), rows.tolist()):
        u = int(cols[i])
        assert (deg[v], v) < (deg[u], u)
        a, b = cols[off[v]:off[v + 1]], cols[off[u]:off[u + 1]]
        assert int(pe[i]) == len(np.intersect1d(a, b, assume_unique=True)), (v, u)
    for v in rng.integers(0, spec.n, 20000).tolist():
        assert np.all(np.diff(cols[off[v]:off[v + 1]]) > 0)
