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
