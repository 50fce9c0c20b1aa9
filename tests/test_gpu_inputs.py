"""Interleaved-pair input (tc_build_pairs) and counting several built graphs at once
(tc_count_graphs), through the C ABI, against tc_build / tc_count and the oracle (exact)."""
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


def _cl(n, seed):
    import graphgen
    s, d = graphgen.chung_lu(n, 2.1, 16.0, 2000.0, 8 * n, seed)
    return n, s, d


@pytest.mark.parametrize("kind", ["pageable", "pinned", "device"])
def test_build_pairs_matches_build(kind):
    n, s, d = _cl(50000, 41)
    pairs = np.stack([s, d], axis=1).copy()
    e = torch.from_numpy(pairs)
    if kind == "pinned":
        e = e.pin_memory()
    elif kind == "device":
        e = e.cuda()
    want = oracle.count_edges(n, s, d)
    with tc.Graph.build_pairs(pairs if kind == "pageable" else e, n) as g, tc.Graph.build(s, d, n) as h:
        assert g.count() == want == h.count()
        _, o1, c1, _ = g.csr()
        _, o2, c2, _ = h.csr()
        assert torch.equal(o1, o2) and torch.equal(c1, c2)


def test_build_pairs_edges_cases():
    with tc.Graph.build_pairs(np.zeros((0, 2), np.int32), 5) as g:
        assert g.count() == 0
    n, s, d = F.complete(30)
    pairs = np.stack([s, d], axis=1).copy()
    pairs[7, 1] = n  # an id outside [0, n)
    with pytest.raises(_lib.TcError) as e:
        tc.Graph.build_pairs(pairs, n)
    assert e.value.code == _lib.TC_ERR_VERTEX_RANGE
    with pytest.raises(_lib.TcError) as e:
        tc.Graph.build_pairs(np.stack([s, d], axis=1), n, options=tc.default_options(hbm_budget_bytes=1024))
    assert e.value.code == _lib.TC_ERR_BUDGET


def test_count_graphs_one_synchronisation():
    gs = []
    want = []
    for j, (n, s, d) in enumerate([_cl(20000, 42), F.wheel(700), F.complete(40), (9, np.zeros(0, np.int32),
                                                                                   np.zeros(0, np.int32)),
                                   _cl(80000, 43)]):
        gs.append(tc.Graph.build(s, d, n))
        want.append(oracle.count_edges(n, s, d))
    try:
        assert tc.count_graphs(gs) == want
        # repeated handles, any order
        order = [4, 0, 4, 2, 0, 1, 3]
        assert tc.count_graphs([gs[j] for j in order]) == [want[j] for j in order]
        assert tc.count_graphs([]) == []
        assert [g.count() for g in gs] == want
    finally:
        for g in gs:
            g.free()
