"""The multi-GPU paths of bench.py: replicas (every rank counts its own copy of the workload
and the ranks meet only to time the slowest one) and a cost-partitioned count (the ranks'
partial counts are summed once).  These tests run that host-side logic as gloo ranks on the
CPU (no GPU is used)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    r, w, local = bench.dist_env()
    pg = bench.init_replicas(w)
    pg.barrier()
    m = bench.max_over_ranks(pg, times[r])
    v = bench.replica_throughput(w, 5, 1000, m)
    total = bench.sum_over_ranks(pg, (1 << 40) + r)  # partial counts beyond 32 bits add exactly
    pg.barrier()
    out.put((r, local, m, v, total))
    pg.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slowest_rank_sets_the_whole_job_throughput(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [100.0 + 50.0 * r for r in range(world)]
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    slowest = max(times)
    for r, local, m, v, total in res:
        assert local == r
        assert m == slowest
        assert total == world * (1 << 40) + sum(range(world))
        # world ranks x 5 steps x 1000 units in the slowest rank's time
        assert v == pytest.approx(world * 5 * 1000 / (slowest / 1e3))


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.init_replicas(1) is None
    assert bench.max_over_ranks(None, 12.5) == 12.5
    assert bench.replica_throughput(1, 4, 10, 20.0) == pytest.approx(2000.0)
    assert bench.sum_over_ranks(None, 7) == 7


def _surrogate_worker(rank, world, port, out):
    """A rank of the partitioned non-overlapping count: its receiving parts of the table, with
    the oracle standing in for the GPU count, summed over the ranks."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import graphgen
    import oracle
    n = 3000
    s, d = graphgen.chung_lu(n, 2.1, 12.0, 600.0, 24_000, 9)
    csr = oracle.oriented_csr(oracle.simple_graph(n, s, d))
    cuts = oracle.balanced_cuts(oracle.vertex_cost(csr, oracle.COST_NEW), 2 * world + 1)
    lo, hi = bench.surrogate_part_range(world, rank, len(cuts) - 1)
    part = int(oracle.count_parts(csr, cuts)[:, lo:hi].sum())
    r, w, _ = bench.dist_env()
    pg = bench.init_replicas(w)
    total = bench.sum_over_ranks(pg, part)
    pg.barrier()
    out.put((r, lo, hi, total, oracle.count(csr)))
    pg.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_partition_ranges_of_the_ranks_add_up(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_surrogate_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # the ranks' ranges tile [0, P) in order, and the partial counts sum to T
    assert res[0][1] == 0 and res[-1][2] == 2 * world + 1
    assert all(a[2] == b[1] for a, b in zip(res, res[1:]))
    for _, _, _, total, T in res:
        assert total == T


def test_part_ranges_cover_every_part_once():
    sys.path.insert(0, ROOT)
    import bench
    for world in range(1, 9):
        for P in range(0, 40):
            got = [bench.surrogate_part_range(world, r, P) for r in range(world)]
            assert got[0][0] == 0 and got[-1][1] == P
            assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
            assert all(0 <= hi - lo - P // world <= 1 for lo, hi in got)
