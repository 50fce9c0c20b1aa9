"""Sanity of the seeded input generators (they hold no counting arithmetic)."""
import os

import numpy as np
import pytest

import graphgen
from graphgen import families as F
from graphgen import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, v = line.split()
            out[k] = v
    return out


def test_er_distinct_pairs_and_determinism():
    s, d = graphgen.erdos_renyi(1000, 20000, 7)
    assert len(s) == 20000 and s.dtype == np.int32
    assert np.all(s != d) and s.min() >= 0 and d.max() < 1000
    key = np.minimum(s, d).astype(np.int64) * 1000 + np.maximum(s, d)
    assert len(np.unique(key)) == 20000
    s2, d2 = graphgen.erdos_renyi(1000, 20000, 7)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)
    s3, _ = graphgen.erdos_renyi(1000, 20000, 8)
    assert not np.array_equal(s, s3)
    with pytest.raises(ValueError):
        graphgen.erdos_renyi(10, 46, 0)  # more than C(10,2) pairs


def test_ba_structure():
    n, k = 5000, 7
    s, d = graphgen.barabasi_albert(n, k, 3)
    assert len(s) == k * (n - k)
    assert np.all(d < s)  # every edge joins a new vertex to an earlier one
    key = s.astype(np.int64) * n + d
    assert len(np.unique(key)) == len(key)
    deg = np.bincount(np.concatenate([s, d]), minlength=n)
    assert deg[k:].min() >= k
    assert deg.max() > 20 * k  # heavy tail


def test_chung_lu_weights_and_draws():
    w = graphgen.chung_lu_weights(100000, 2.1, 40.0, 5000.0)
    assert abs(w.mean() - 40.0) < 1e-6
    assert np.all(np.diff(w) <= 0)
    assert 0.8 * 5000 < w[0] < 1.25 * 5000
    s, d = graphgen.chung_lu(100000, 2.1, 40.0, 5000.0, 2_000_000, 9)
    assert s.min() >= 0 and max(s.max(), d.max()) < 100000
    deg = np.bincount(np.concatenate([s, d]), minlength=100000)
    assert abs(deg[0] - w[0]) < 6 * np.sqrt(w[0]) + 1
    s2, d2 = graphgen.chung_lu(100000, 2.1, 40.0, 5000.0, 2_000_000, 9)
    assert np.array_equal(s, s2) and np.array_equal(d, d2)


def test_workload_specs():
    assert W.ER_10K.num_input_edges == 100_000
    assert W.BA_1M.num_input_edges == 49_997_500
    assert W.CL_10M.num_input_edges == 200_000_000
    specs = W.batch_specs(64)
    assert [s.family for s in specs[:4]] == ["er", "ba", "er", "ba"]
    for s in specs:
        assert 1000 <= s.n <= 200_000
    sv = W.serve_spec(3)
    assert sv.family == "cl" and 10_000 <= sv.n <= 2_000_000 and 2.1 <= sv.gamma <= 2.8
    t = W.poisson_arrivals(2000, 2000.0)
    assert np.all(np.diff(t) > 0) and 0.7 < t[-1] < 1.3


def test_golden_er_graph_is_reproduced():
    """The integer-only ER generator reproduces the stored graph on any platform."""
    import hashlib
    import oracle
    g = read_golden("er_10k.txt")
    s, d = W.ER_10K.edges()
    csr = oracle.oriented_csr(oracle.simple_graph(W.ER_10K.n, s, d))
    assert csr.m_hat == int(g["m_hat"])
    assert hashlib.sha256(csr.cols.astype("<i4").tobytes()).hexdigest() == g["sha256_cols"]
    assert oracle.count(csr) == int(g["triangles"])


def test_families_shapes():
    n, s, d = F.wheel(6)
    assert n == 6 and len(s) == 10
    n, s, d = F.complete_tripartite(1, 2, 3)
    assert n == 6 and len(s) == 2 + 3 + 6
    n, s, d = F.disjoint_union(F.cycle(3), F.cycle(4))
    assert n == 7 and s.max() == 6
