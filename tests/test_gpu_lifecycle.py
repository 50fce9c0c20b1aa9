"""Handles under concurrent callers and repeated use: threads counting different graphs on
their own streams get exact totals, and build / count / free cycles of graphs, batches and
servers leave device memory where it was."""
import threading

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


def _graphs():
    gs = []
    for j in range(8):
        sp = W.serve_spec(j, seed=55, n_lo=5000, n_hi=80000, d_lo=8, d_hi=40)
        s, d = sp.edges()
        gs.append((s, d, sp.n))
    return gs


GRAPHS = _graphs()
WANT = [oracle.count_edges(n, s, d) for s, d, n in GRAPHS]


def test_threads_count_concurrently_on_their_own_streams():
    errors, got = [], {}

    def work(tid):
        try:
            torch.cuda.set_device(0)
            stream = torch.cuda.Stream()
            for rep in range(3):
                j = (tid + rep) % len(GRAPHS)
                s, d, n = GRAPHS[j]
                with tc.Graph.build(s, d, n, stream=stream) as g:
                    got[(tid, rep)] = (j, g.count(stream), g.count_partition(1, 2, stream) + g.count_partition(0, 2, stream))
        except Exception as e:  # pragma: no cover - reported below
            errors.append(repr(e))

    threads = [threading.Thread(target=work, args=(t,)) for t in range(6)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=300)
    assert not errors, errors
    assert len(got) == 18
    for (tid, rep), (j, T, T2) in got.items():
        assert T == WANT[j] and T2 == WANT[j], (tid, rep, j)


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def test_repeated_cycles_do_not_grow_device_memory():
    s, d, n = GRAPHS[0]

    def cycle():
        with tc.Graph.build(s, d, n) as g:
            g.count()
            T, tv = g.count_per_vertex()
            del tv
        with tc.Batch.build(GRAPHS[:4]) as b:
            b.count()
        with tc.Server(4 << 30, slots=2) as sv:
            for j in range(4):
                sv.submit(*GRAPHS[j])
            sv.drain(120_000)
            sv.poll()

    for _ in range(3):  # reach the pools' steady state
        cycle()
    before = _free_bytes()
    for _ in range(20):
        cycle()
    after = _free_bytes()
    assert before - after < 64 << 20, (before, after)  # no growth beyond allocator granularity
