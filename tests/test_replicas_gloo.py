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
