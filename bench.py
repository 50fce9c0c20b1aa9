#!/usr/bin/env python
"""Benchmark of the GB300 exact triangle counter.

One step = one pass of the whole path over the workload's edge list: build (canonical
keys, radix sort, dedupe, degrees, orientation, N+ lists, tasks) and count (cost prefix,
Eq. 1 / Eq. 2 schedule, persistent intersection kernel, exact reduction), through the C ABI.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload cl|ba|er] [--impl gb300|reference]

Prints one JSON line (rank 0).  `value` is oriented edges (distinct undirected edges) per
second over all ranks with the edge list resident in HBM when the timed region starts;
`e2e` is the same metric with the edge list in pinned host memory, copies included.
With N > 1 every rank counts its own replica of the workload (replicas only: the
counts need no exchange), so the scaling is weak.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "exact oriented-edges/s per GB300"
UNIT = "oriented-edges/s"
FALLBACK_HBM_GBS = 6800.0
WORKLOAD_TEXT = {
    "cl": "chung-lu n=10,000,000 exponent 2.1 mean degree 40 w0=1e5, 2.0e8 edge draws, seed 2",
    "ba": "barabasi-albert n=1,000,000 k=50 (avg degree 100), seed 1",
    "er": "erdos-renyi G(n=10,000, m=100,000), seed 0",
    "cl_small": "chung-lu n=2,000,000 exponent 2.1 mean degree 40 w0=44,721, 4.0e7 edge draws, seed 2 (profiling size)",
    "cl_twitter": "chung-lu n=41,650,000 exponent 2.1 mean degree 115 w0=3e6, 2.4e9 edge draws, seed 5 "
                  "(the size of the paper's Twitter graph)",
}
# input pairs of the prefix the CPU baseline also times on one core, end to end
CPU_SAMPLE_PAIRS = {"cl": 32_000_000, "ba": 16_000_000, "er": 100_000, "cl_small": 8_000_000, "cl_twitter": 32_000_000}
# input pairs per step of the reference (oracle) arm, so that --steps K --warmup W ends in minutes
REF_SAMPLE_PAIRS = {"cl": 4_000_000, "ba": 2_000_000, "er": 100_000, "cl_small": 2_000_000, "cl_twitter": 4_000_000}
REF_BATCH_GRAPHS = 8
REF_SERVE_GRAPHS = 2


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--workload", default="cl", choices=["cl", "ba", "er", "cl_small", "cl_twitter", "batch", "serve"])
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-batch", action="store_true", help="skip the batched-vs-plain leg")
    p.add_argument("--no-serve", action="store_true", help="skip the serving-vs-plain leg")
    p.add_argument("--no-per-vertex", action="store_true",
                   help="skip the per-vertex / per-edge / clustering timings of the optional outputs")
    p.add_argument("--pack-edges", type=int, default=0, help="input edges per batch pack (0: the library default)")
    p.add_argument("--partitioned", action="store_true",
                   help="one graph split over the ranks: every rank builds it and counts its cost-balanced "
                        "part of the tasks; the partial counts are summed (strong scaling)")
    p.add_argument("--partition-mode", default="tasks", choices=["tasks", "surrogate"],
                   help="with --partitioned: split the cost-ordered tasks of a replica (tasks), or give each "
                        "rank its receiving parts of Sec. IV's non-overlapping partition of the lists, read from "
                        "page-locked host memory (surrogate)")
    p.add_argument("--ablation", action="store_true",
                   help="count the workload under every cost model and static share of Eq. 1 and print one "
                        "JSON line per setting (kernel times and per-worker idle spread)")
    p.add_argument("--serve-requests", type=int, default=0,
                   help="requests of the serving window (default 2000)")
    p.add_argument("--serve-slots", type=int, default=4, help="slot threads of the server")
    p.add_argument("--serve-group-edges", type=int, default=0, help="input edges one slot takes at once (0: default)")
    p.add_argument("--serve-pool", type=int, default=0,
                   help="pre-generated graphs the requests cycle through (default 256)")
    p.add_argument("--no-surrogate", action="store_true",
                   help="skip the leg that counts the lists over a non-overlapping partition (Sec. IV) from "
                        "page-locked host memory")
    p.add_argument("--surrogate-fraction", type=int, default=4,
                   help="the part-size bound of that leg, as a fraction of the lists (default 4: each part "
                        "holds at most a quarter of them)")
    p.add_argument("--batch-graphs", type=int, default=0,
                   help="graphs of the batched workload (default 4096)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# Replicas: with N > 1 every rank counts its own copy of the workload on its own GPU.  The
# counts need no exchange; the ranks only meet at barriers around the timed region and to
# take the slowest rank's time.  A gloo group carries those few host-side messages.

def init_replicas(world):
    """The process group of the replicas (None for one process)."""
    if world <= 1:
        return None
    import torch.distributed as dist
    if not dist.is_initialized():
        dist.init_process_group("gloo")
    return dist


def max_over_ranks(pg, x):
    """The largest value of x over all ranks (x itself for one process)."""
    if pg is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, x):
    """The exact sum of the integer x over all ranks (the one reduction of a partitioned count)."""
    if pg is None:
        return int(x)
    import torch
    t = torch.tensor([int(x)], dtype=torch.int64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return int(t.item())


def replica_throughput(world, steps, units_per_step, max_ms):
    """Whole-job throughput: units all ranks processed over the slowest rank's time."""
    return world * steps * units_per_step / (max_ms / 1e3)


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while running (start before, stop after the timed region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: str | None):
        self.lines = []
        self.proc = None
        self.gpu_index = gpu_index

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_index is not None:
            cmd += ["-i", self.gpu_index]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- helpers

def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def count_kernel_source_hash():
    with open(os.path.join(ROOT, "paper_1406_5687_gb300", "csrc", "count.cu"), "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def stored_traffic(workload):
    """DRAM bytes (read + write) per launch of k_count_big from a committed ncu summary, if
    it is still about the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"k_count_big_{workload}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if rec.get("count_cu_sha256") != count_kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def stored_surrogate_traffic():
    """DRAM bytes (read + write) of k_surrogate_count over the parts of one host-list call of the
    bench's surrogate leg, from the ncu capture in profiles/, or None when surrogate.cu has changed
    since it was taken."""
    path = os.path.join(ROOT, "profiles", "k_surrogate_count_cl_traffic.json")
    src = os.path.join(ROOT, "paper_1406_5687_gb300", "csrc", "surrogate.cu")
    try:
        rec = json.load(open(path))
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except (OSError, ValueError):
        return None
    return rec.get("dram_bytes_per_call") if rec.get("surrogate_cu_sha256") == sha else None


def algorithmic_bytes(g, opt):
    """Bytes the count kernels must move per count if nothing were cached, per class.

    Every task reads its 16-byte record and the partner-list entries its kernel must test:
    a small owner's partner list whole; for a big owner, only the part inside the owner
    list's [first, last] range (both lists are ascending), found with the list's first and
    last entry (8 bytes) and a binary search.  Every owner's list is staged once (4 B per
    entry) with its two offsets (16 B), a big owner also reading its first and last entry
    (8 B).  The entries read are counted by the kernels themselves in one traced count
    (`streamed`).  Also returns the merge-direction figure 4 (sum_{(v,u)} |N+(u)| + m_hat)
    + 16 n of the paper's Fig. 1."""
    import numpy as np
    _, meta, _, _ = g.count_ex(opt, streamed=True)
    streamed = meta["streamed"]
    deg, off, cols, tasks = g.csr()
    off = off.cpu().numpy()
    owner = tasks[:, 0].cpu().numpy()
    dh = np.diff(off)
    info = g.info()
    ts = int(info["tasks_small"])

    def part(lo, hi, cls):
        owners = np.unique(owner[lo:hi])
        nt = hi - lo
        b = 16 * nt + 4 * streamed[cls] + 4 * int(dh[owners].sum()) + 16 * len(owners)
        if cls == 1:
            b += 8 * nt + 8 * len(owners)
        return {"bytes": int(b), "streamed_entries": int(streamed[cls]), "owners": int(len(owners)), "tasks": int(nt)}

    small, big = part(0, ts, 0), part(ts, len(owner), 1)
    b_merge = 4 * (int(info["sum_dhat_u"]) + int(info["m_hat"])) + 16 * int(info["n"])
    return {"small": small, "big": big, "total": small["bytes"] + big["bytes"], "merge": b_merge,
            "untrimmed_big_entries": int(info["sum_stream"]) - int(streamed[0])}


def _bits_for(x):
    """Bits of the largest id below x (at least 1), as the library sizes its keys."""
    return max(1, int(x - 1).bit_length()) if x > 1 else 1


def build_bytes(info):
    """Compulsory DRAM bytes of one build (steps a1-a5 and the task array), counting each
    streamed array access once and the random-access arrays (degrees, offsets, numbering) once
    by their size: k_canon reads 8 and writes 8 per input pair; every onesweep pass reads and
    writes 8 per key (the 48-bit edge keys: 2b bits, the oriented keys: the b owner bits, the
    task keys: bits(n + 1)); the dedupe pass and the orienting compaction read the sorted keys
    (8 each) and write 8 per distinct edge; the lists' last pass also writes cols (4); the task
    keys read 8 and write 8 per oriented edge; the task sort's last pass writes 16-byte records
    instead of keys and each big owner's first task at its owner number; the owner index clears
    that array of n + 1 numbers (4 each) and compacts it (read twice)."""
    m, mh, T, n = int(info["m_input"]), int(info["m_hat"]), int(info["tasks"]), int(info["n"])
    b = _bits_for(n)
    p1, p2, p3 = -(-2 * b // 8), -(-b // 8), -(-_bits_for(n + 1) // 8)
    terms = {
        "canon": 16 * m,
        "sort_edges": 16 * p1 * m,
        "dedupe_degree": 8 * m + 8 * n,
        "orient_compact": 8 * m + 8 * mh + 4 * n,
        "sort_lists": 16 * p2 * mh + 4 * mh,
        "offsets": 4 * n + 8 * (n + 1),
        "task_keys": 16 * mh + 12 * n,
        "sort_tasks": 16 * (p3 - 1) * mh + 8 * mh + 16 * T + 8 * (n + 1) + 4 * n,
        "owner_index": 12 * (n + 1),
    }
    return {"bytes": sum(terms.values()), "terms": terms, "sort_passes": [p1, p2, p3],
            "sort_bytes": 16 * (p1 * m + (p2 + p3) * mh)}


def cpu_baseline(workload, sample_pairs, single_thread_budget_s=60.0):
    """The oracle as it stands (simple graph, Fig. 1 lists, Fig. 1 count) on the whole benched
    graph, timed on the host: the simple graph and the lists as the oracle builds them (one
    thread), then the count loop with the oracle's OpenMP option on every host core.  The value
    is m_hat over that end-to-end time.  Beside it: the count loop alone on all cores and, when
    the all-core time says it fits `single_thread_budget_s`, on one core (the same CSR); and the
    older single-thread figure on the first `sample_pairs` input pairs."""
    import oracle
    from graphgen import workloads as W
    spec = W.SINGLE[workload]
    cores = os.cpu_count() or 1
    s, d = spec.edges()
    t0 = time.perf_counter()
    csr = oracle.oriented_csr(oracle.simple_graph(spec.n, s, d))
    t1 = time.perf_counter()
    T = oracle.count(csr, threads=cores)
    t2 = time.perf_counter()
    build_s, count_s = t1 - t0, t2 - t1
    out = {"value": csr.m_hat / (t2 - t0), "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"the whole benched graph ({len(s):,} input pairs, {csr.m_hat:,} distinct edges, {T:,} triangles): "
                     f"the oracle's simple graph and Fig. 1 lists on one thread ({build_s:.2f} s), then its Fig. 1 "
                     f"count loop with OpenMP over all {cores} host cores ({count_s:.2f} s)",
           "seconds": t2 - t0, "build_seconds": build_s, "triangles": T,
           "count_only_all_cores": {"value": csr.m_hat / count_s, "cores": cores, "seconds": count_s}}
    if count_s * cores <= single_thread_budget_s:
        t3 = time.perf_counter()
        T1 = oracle.count(csr, threads=1)
        c1 = time.perf_counter() - t3
        if T1 != T:
            raise RuntimeError("oracle count differs between thread counts")
        out["count_only_one_core"] = {"value": csr.m_hat / c1, "cores": 1, "seconds": c1}
    else:
        out["count_only_one_core"] = {"value": None, "cores": 1,
                                      "note": f"not run: about {count_s * cores:.0f} s expected (all-core time x "
                                              f"{cores} cores), over the bench's {single_thread_budget_s:.0f} s bound"}
    del csr, s, d
    # the single-thread end-to-end figure on a prefix of the same workload
    if spec.family == "cl":
        import dataclasses
        s, d = dataclasses.replace(spec, draws=min(sample_pairs, spec.draws)).edges()
    else:
        s, d = spec.edges()
        s, d = s[:sample_pairs], d[:sample_pairs]
    t4 = time.perf_counter()
    c2 = oracle.oriented_csr(oracle.simple_graph(spec.n, s, d))
    oracle.count(c2, threads=1)
    dt = time.perf_counter() - t4
    out["one_core_prefix"] = {"value": c2.m_hat / dt, "cores": 1, "seconds": dt,
                              "sample": f"first {len(s):,} input pairs ({c2.m_hat:,} distinct edges), end to end"}
    return out


# --------------------------------------------------------------------------- batched and plain

BATCH_TEXT = ("batched: graphs of the 4096-graph workload, seed 3 (even index Erdos-Renyi, odd index "
              "Barabasi-Albert; n log-uniform in [1e3, 2e5]; average degree uniform in [8, 128])")


def batch_inputs(count, threads=None):
    """The first `count` graphs of the batched workload, generated in parallel, each edge list
    in pinned host memory: [(src, dst, n)]."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from graphgen import workloads as W
    specs = W.batch_specs(count)

    def gen(sp):
        s, d = sp.edges()
        return torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory(), sp.n

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 4) as ex:
        return list(ex.map(gen, specs))


def batch_leg(count, steps, warmup, tune_sample=64, oracle_sample=4, pack_edges=0):
    """Batched counting of `count` graphs against the plain per-graph path on the same GPU.

    batched: tc_batch_build + tc_batch_run per step (edge lists resident in HBM, then from
    pinned host memory for e2e); plain: tc_build + tc_count + tc_free per graph.  Both use the
    options the autotuner picks on the first `tune_sample` graphs."""
    import numpy as np
    import torch
    import paper_1406_5687_gb300 as tc
    t0 = time.perf_counter()
    host = batch_inputs(count)
    gen_s = time.perf_counter() - t0
    dev = [(s.cuda(non_blocking=True), d.cuda(non_blocking=True), n) for s, d, n in host]
    torch.cuda.synchronize()
    m_in = sum(int(s.numel()) for s, _, _ in host)
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    best, rep = tc.autotune(dev[:tune_sample], reps=2, stream=stream)
    tune_s = time.perf_counter() - t0
    chosen = {k: getattr(best, k) for k in ("small_max", "warps_per_block", "big_warps", "piece", "static_percent")}

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # batched, edge lists resident in HBM: build + count per step
    def batched_step(graphs):
        e0, e1, e2 = ev(), ev(), ev()
        e0.record(stream)
        b = tc.Batch.build(graphs, options=best, pack_edges=pack_edges, stream=stream)
        e1.record(stream)
        out = torch.empty(count, dtype=torch.int64, device="cuda")
        b.run(out, stream)
        e2.record(stream)
        b.check(stream)
        e2.synchronize()
        info = b.info()
        b.free()
        return e0.elapsed_time(e2), e0.elapsed_time(e1), e1.elapsed_time(e2), out, info

    for _ in range(warmup):
        batched_step(dev)
    l0 = tc.kernel_launches()
    res = [batched_step(dev) for _ in range(steps)]
    launches = (tc.kernel_launches() - l0) // steps
    totals = res[-1][3].cpu().numpy().astype(np.uint64)
    info = res[-1][4]
    b_ms = statistics.mean(r[0] for r in res)
    b_build = statistics.mean(r[1] for r in res)
    b_count = statistics.mean(r[2] for r in res)

    # count only, CSR resident: replays of the captured launch
    b = tc.Batch.build(dev, options=best, pack_edges=pack_edges, stream=stream)
    out = torch.empty(count, dtype=torch.int64, device="cuda")
    for _ in range(warmup):
        b.run(out, stream)
    e0, e1 = ev(), ev()
    e0.record(stream)
    for _ in range(steps):
        b.run(out, stream)
    e1.record(stream)
    b.check(stream)
    replay_ms = e0.elapsed_time(e1) / steps
    if not np.array_equal(out.cpu().numpy().astype(np.uint64), totals):
        raise RuntimeError("batched totals changed between runs")
    edges = b.graph_edges()
    b.free()

    # e2e: edge lists in pinned host memory, the k totals read back to the host
    def batched_host():
        t = time.perf_counter()
        bb = tc.Batch.build(host, options=best, pack_edges=pack_edges, stream=stream)
        got = bb.count(stream)
        bb.free()
        return (time.perf_counter() - t) * 1e3, got
    batched_host()
    e2e = [batched_host() for _ in range(steps)]
    if not np.array_equal(e2e[-1][1], totals):
        raise RuntimeError("batched e2e totals differ")
    e2e_ms = statistics.mean(x[0] for x in e2e)

    # plain: one graph at a time through tc_build + tc_count, same options
    def plain_pass(graphs):
        tot = np.zeros(count, np.uint64)
        cnt_ms = 0.0
        torch.cuda.synchronize()
        t = time.perf_counter()
        for j, (s, d, n) in enumerate(graphs):
            g = tc.Graph.build(s, d, n, best, stream=stream)
            c0 = time.perf_counter()
            tot[j] = g.count(stream)
            cnt_ms += (time.perf_counter() - c0) * 1e3
            g.free()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) * 1e3, cnt_ms, tot
    plain_pass(dev[:min(count, 64)])
    p_ms, p_count_ms, p_tot = plain_pass(dev)
    p_host_ms, _, _ = plain_pass(host)
    if not np.array_equal(p_tot, totals):
        raise RuntimeError("plain and batched totals differ")

    # the oracle on a few of the graphs, one by one
    import oracle
    picks = list(range(0, count, max(1, count // oracle_sample)))[:oracle_sample]
    for j in picks:
        s, d, n = host[j]
        want = oracle.count_edges(n, s.numpy(), d.numpy())
        if want != int(totals[j]):
            raise RuntimeError(f"graph {j}: batched {int(totals[j])} != oracle {want}")
    return {
        "workload": BATCH_TEXT, "graphs": count, "m_input": m_in, "m_hat": int(edges.sum()),
        "packs": info["packs"], "triangles": int(totals.sum()), "unit": "graphs/s",
        "batched": {"graphs_per_s": count / (b_ms / 1e3), "ms": b_ms, "build_ms": b_build, "count_ms": b_count,
                    "count_only_graphs_per_s": count / (replay_ms / 1e3), "replay_ms": replay_ms,
                    "e2e_graphs_per_s": count / (e2e_ms / 1e3), "e2e_ms": e2e_ms, "gpu_launches_per_step": launches},
        "plain": {"graphs_per_s": count / (p_ms / 1e3), "ms": p_ms,
                  "count_only_graphs_per_s": count / (p_count_ms / 1e3), "count_ms": p_count_ms,
                  "e2e_graphs_per_s": count / (p_host_ms / 1e3), "e2e_ms": p_host_ms},
        "speedup": {"build_and_count": p_ms / b_ms, "count_only": p_count_ms / replay_ms, "e2e": p_host_ms / e2e_ms},
        "autotune": {"sample_graphs": min(tune_sample, count), "tried": rep["tried"], "chosen": chosen,
                     "best_ms": rep["best_ms"], "default_ms": rep["default_ms"], "seconds": tune_s},
        "oracle_checked_graphs": picks, "generate_s": gen_s,
        "timing": "batched: CUDA events on the launching stream; plain: host wall clock around each "
                  "synchronous call (the plain path returns each total to the host)",
    }


# --------------------------------------------------------------------------- serving and plain

SERVE_TEXT = ("serving: Poisson arrivals at 2,000 graphs/s of Chung-Lu graphs, seed 4 (exponent uniform in "
              "[2.1, 2.8], n log-uniform in [1e4, 2e6], average degree uniform in [16, 96]), a finite window of "
              "requests cycling through a pool of pre-generated graphs in pinned host memory, 60 GB budget")
SERVE_RATE = 2000.0
SERVE_BUDGET = 60 << 30


def serve_pool(count):
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from graphgen import workloads as W

    def gen(j):
        sp = W.serve_spec(j)
        s, d = sp.edges()
        return torch.from_numpy(s).pin_memory(), torch.from_numpy(d).pin_memory(), sp.n

    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return list(ex.map(gen, range(count)))


def _pct(x, q):
    import numpy as np
    return float(np.percentile(np.asarray(x), q)) * 1e3


def serve_leg(requests, pool_size, slots=4, group_edges=0):
    """The server (continuous batching, `slots` slot threads, 60 GB budget) against a
    one-at-a-time loop of tc_build + tc_count + tc_free, on the same Poisson arrival trace."""
    import numpy as np
    import torch
    import paper_1406_5687_gb300 as tc
    from graphgen import workloads as W
    t0 = time.perf_counter()
    pool = serve_pool(pool_size)
    gen_s = time.perf_counter() - t0
    arrivals = W.poisson_arrivals(requests, SERVE_RATE)
    pick = [i % pool_size for i in range(requests)]
    edges_in = sum(int(pool[j][0].numel()) for j in pick)

    with tc.Server(SERVE_BUDGET, slots=slots, group_edges=group_edges) as sv:
        for j in range(min(4, pool_size)):  # warm-up
            sv.submit(*pool[j], tag=-1)
        sv.drain(-1)
        sv.poll(16)
        l0 = tc.kernel_launches()
        start = time.perf_counter()
        for i in range(requests):
            delay = start + arrivals[i] - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            sv.submit(*pool[pick[i]], tag=i)
        sv.drain(-1)
        res = sorted(sv.poll(requests + 16), key=lambda r: r["tag"])
        launches = tc.kernel_launches() - l0
        st = sv.stats()
    if len(res) != requests or any(r["status"] != 0 for r in res):
        raise RuntimeError("serving lost or failed requests")
    s_lat = [r["t_done"] - r["t_submit"] for r in res]
    s_span = max(r["t_done"] for r in res) - min(r["t_submit"] for r in res)
    s_tot = [r["total"] for r in res]

    # plain: one request at a time on the same arrival trace
    stream = torch.cuda.current_stream()
    p_lat, p_tot = [], []
    for j in range(min(4, pool_size)):
        g = tc.Graph.build(*pool[j][:2], pool[j][2], stream=stream)
        g.count(stream)
        g.free()
    start = time.perf_counter()
    for i in range(requests):
        arrive = start + arrivals[i]
        delay = arrive - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        s_, d_, n_ = pool[pick[i]]
        g = tc.Graph.build(s_, d_, n_, stream=stream)
        p_tot.append(g.count(stream))
        g.free()
        p_lat.append(time.perf_counter() - arrive)
    p_span = time.perf_counter() - start
    if p_tot != s_tot:
        raise RuntimeError("served totals differ from the plain path")
    import oracle
    for j in range(min(2, pool_size)):
        s_, d_, n_ = pool[j]
        if oracle.count_edges(n_, s_.numpy(), d_.numpy()) != s_tot[j]:
            raise RuntimeError(f"request {j}: served total differs from the oracle")
    return {
        "workload": SERVE_TEXT, "requests": requests, "pool_graphs": pool_size, "edges_in": edges_in,
        "offered_graphs_per_s": SERVE_RATE, "slots": slots, "unit": "graphs/s",
        "served": {"graphs_per_s": requests / s_span, "edges_per_s": edges_in / s_span,
                   "p50_ms": _pct(s_lat, 50), "p99_ms": _pct(s_lat, 99), "span_s": s_span,
                   "groups": st["groups"], "grouped_requests": st["grouped"],
                   "peak_bytes_in_flight": st["peak_bytes_in_flight"], "peak_slots_busy": st["peak_slots_busy"],
                   "gpu_launches": launches},
        "plain": {"graphs_per_s": requests / p_span, "edges_per_s": edges_in / p_span,
                  "p50_ms": _pct(p_lat, 50), "p99_ms": _pct(p_lat, 99), "span_s": p_span},
        "p99_vs_plain": _pct(s_lat, 99) / _pct(p_lat, 99),
        "throughput_vs_plain": p_span / s_span,
        "oracle_checked_requests": list(range(min(2, pool_size))), "generate_s": gen_s,
        "latency": "arrival (submit) to result on the host, steady clock",
    }


# --------------------------------------------------------------------------- reference arm

def surrogate_leg(s_dev, d_dev, n, opt, T_ref, stream, fraction=4, reps=3):
    """Sec. IV's count over a non-overlapping partition (tc_count_surrogate) of the workload's N+
    lists held in page-locked host memory: no more than 1/fraction of the lists is in device memory
    at once (two part slices).  Cuts from tc_surrogate_plan with equal list entries per part.  Each
    call is timed with CUDA events on the stream it runs on (it synchronises that stream), the best
    of `reps` after one warm-up; the same cuts over device-resident lists and the work-balanced cuts
    of Sec. IV-F are timed beside it."""
    import numpy as np
    import torch
    import paper_1406_5687_gb300 as tc

    gg = tc.Graph.build(s_dev, d_dev, n, opt)
    _, off, cols, _ = gg.csr()
    gg.free()
    m = int(cols.numel())
    off_h, cols_h = off.cpu().pin_memory(), cols.cpu().pin_memory()
    budget = max(4 * m // fraction, 1)
    t0 = time.perf_counter()
    cuts = tc.surrogate_plan(off_h, cols_h, part_bytes=budget, fn=tc.TC_FN_LIST)
    plan_ms = (time.perf_counter() - t0) * 1e3
    o = off_h.numpy()
    slices = o[cuts[1:]] - o[cuts[:-1]]

    def timed(of, co, cu):
        best = None
        for k in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            T, _tab = tc.count_surrogate(of, co, cu, stream=stream)
            e1.record(stream)
            e1.synchronize()
            if T != T_ref:
                raise RuntimeError(f"surrogate count {T} != {T_ref}")
            if k > 0:
                ms = e0.elapsed_time(e1)
                best = ms if best is None or ms < best else best
        return {"ms": best, "value": m / (best / 1e3), "unit": UNIT}

    host = timed(off_h, cols_h, cuts)
    # cuts bounded in work (Sec. IV-F cost, as many parts) and in size (the same byte bound) at once:
    # parts of more even time, for ranks that count parts side by side
    both = tc.surrogate_plan_both(off_h, cols_h, len(cuts) - 1, budget)
    host_both = timed(off_h, cols_h, both)

    def part_times(cu):
        # each receiving part alone (its messages routed and counted), best of 2, CUDA events
        out = []
        for j in range(len(cu) - 1):
            best = None
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                tc.count_surrogate(off_h, cols_h, cu, part_lo=j, part_hi=j + 1, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None or ms < best else best
            out.append(best)
        return {"part_ms": out, "max_over_mean": max(out) / (sum(out) / len(out))}

    parts_equal, parts_both = part_times(cuts), part_times(both)
    bs = o[both[1:]] - o[both[:-1]]
    # one more call with the work counters and per-kernel CUDA events (outside the timed best-of)
    T, _tab, st = tc.count_surrogate(off_h, cols_h, cuts, stream=stream, stats=True)
    if T != T_ref:
        raise RuntimeError("surrogate count with counters disagrees")
    dev = timed(off, cols, cuts)
    one = timed(off, cols, np.array([0, n], np.int32))
    work_cuts = tc.surrogate_plan(off, cols, nparts=len(cuts) - 1, fn=tc.TC_FN_NEW)
    work = timed(off, cols, work_cuts)
    ws = o[work_cuts[1:]] - o[work_cuts[:-1]]
    del off, cols, off_h, cols_h
    torch.cuda.empty_cache()
    # k_surrogate_count's algorithmic bytes per call: per item its 16-byte record and the staged
    # message (4 per entry); per (v, u) pair -- m_hat of them, each oriented edge once -- the entry u
    # (4) and N_u's offsets (16); and the resident entries streamed after trimming (4 each)
    alg = 16 * st["items"] + 4 * st["staged"] + 20 * m + 4 * st["streamed"]
    peak, peak_kind = measured_peaks()
    achieved = alg / (st["count_ms"] / 1e3) / 1e9
    roofline = {"kernel": "k_surrogate_count (SurrogateCount of Fig. 2, all parts of one call)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"hbm_gbs of {peak_kind}", "traffic": stored_surrogate_traffic(),
                "algorithmic_bytes": alg, "kernel_ms": st["count_ms"], "route_ms": st["route_ms"],
                "work": st}
    return {"parts": len(cuts) - 1, "part_bytes_bound": budget, "lists_bytes": 4 * m,
            "largest_part_bytes": int(4 * slices.max()), "plan_ms": plan_ms,
            "host_lists": dict(host, per_part=parts_equal),
            "host_lists_work_and_size_cuts": dict(host_both, parts=len(both) - 1, largest_part_bytes=int(4 * bs.max()),
                                                  per_part=parts_both,
                                                  cuts="tc_surrogate_plan_both: bounded in work (Sec. IV-F cost, "
                                                       "%d parts) and in size (the byte bound) at once" % (len(cuts) - 1)),
            "device_lists": dev, "device_lists_one_part": one,
            "device_lists_work_balanced_cuts": dict(work, largest_part_bytes=int(4 * ws.max())),
            "h2d_bytes_per_count": int(4 * sum(int(o[b]) - (int(o[a]) & ~3) for a, b in zip(cuts[:-1], cuts[1:]))),
            "roofline": roofline,
            "note": "tc_count_surrogate: parts counted one after another, each part's slice copied in "
                    "(the next copy overlapping this count), every list read in place as a message; "
                    "value = m_hat / ms of one call, CUDA events on its stream, best of %d after a warm-up; "
                    "per_part: each receiving part counted alone; h2d_bytes_per_count counts the slice copies "
                    "only (messages are read in place)" % reps}


def run_reference_batch(args):
    """The oracle, graph by graph, on the first graphs of the batched (or served) workload, a
    bounded sample per step: graphs/s on the host."""
    import oracle
    from graphgen import workloads as W
    serve = args.workload == "serve"
    specs = [W.serve_spec(j) for j in range(REF_SERVE_GRAPHS)] if serve else W.batch_specs(REF_BATCH_GRAPHS)
    graphs = [(sp.n,) + sp.edges() for sp in specs]
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        for n, s, d in graphs:
            oracle.count_edges(n, s, d)
        if i >= args.warmup:
            times.append(time.perf_counter() - t0)
    mean = sum(times) / len(times)
    value = len(graphs) / mean
    line = {"impl": "reference", "metric": "served graphs/s" if serve else "batched graphs/s", "value": value,
            "unit": "graphs/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": SERVE_TEXT if serve else BATCH_TEXT, "graphs": len(graphs)},
            "cpu_baseline": {"value": value, "unit": "graphs/s", "cores": 1, "kind": "oracle",
                             "sample": f"first {len(graphs)} graphs of the {'served' if serve else 'batched'} "
                                       "workload per step, oracle end to end, one graph after another, "
                                       "single thread"},
            "e2e": {"value": value, "unit": "graphs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    if args.workload in ("batch", "serve"):
        return run_reference_batch(args)
    import oracle
    from graphgen import workloads as W
    spec = W.SINGLE[args.workload]
    pairs = REF_SAMPLE_PAIRS[args.workload]
    if spec.family == "cl":
        import dataclasses
        s, d = dataclasses.replace(spec, draws=min(pairs, spec.draws)).edges()
    else:
        s, d = spec.edges()
        s, d = s[:pairs], d[:pairs]
    times, mh = [], 0
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        csr = oracle.oriented_csr(oracle.simple_graph(spec.n, s, d))
        oracle.count(csr)
        dt = time.perf_counter() - t0
        mh = csr.m_hat
        if i >= args.warmup:
            times.append(dt)
    mean = sum(times) / len(times)
    value = mh / mean
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": mean * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD_TEXT[args.workload], "sample_pairs": len(s), "m_hat": mh},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {len(s):,} input pairs of the workload per step, "
                                       "oracle end to end, single thread"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- GPU arm

def run_batch_only(args, rank, world, local):
    """--workload batch: the batched leg alone at its full size, as the JSON line's metric."""
    import torch
    torch.cuda.set_device(local)
    pg = init_replicas(world)
    count = args.batch_graphs or 4096
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    leg = batch_leg(count, args.steps, args.warmup, pack_edges=args.pack_edges)
    clk = clocks.stop()
    ms = max_over_ranks(pg, leg["batched"]["ms"])
    if rank == 0:
        b = leg["batched"]
        line = {"metric": "batched graphs/s", "value": replica_throughput(world, 1, count, ms), "unit": "graphs/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": leg["workload"], "graphs": count, "m_input": leg["m_input"],
                           "m_hat": leg["m_hat"], "packs": leg["packs"],
                           "l2": "inputs larger than L2 (edge lists and lists exceed 129 MB)",
                           "parallelism": "replicas" if world > 1 else "single"},
                "roofline": None, "cpu_baseline": None,
                "e2e": {"value": world * count / (b["e2e_ms"] / 1e3), "unit": "graphs/s",
                        "h2d_bytes_per_step": 8 * leg["m_input"], "d2h_bytes_per_step": 8 * count},
                "gpu_launches": b["gpu_launches_per_step"] * args.steps, "clocks": clk, "batch": leg}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_serve_only(args, rank, world, local):
    """--workload serve: the serving leg alone at its full window, as the JSON line's metric."""
    import torch
    torch.cuda.set_device(local)
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    leg = serve_leg(args.serve_requests or 2000, args.serve_pool or 256, args.serve_slots, args.serve_group_edges)
    clk = clocks.stop()
    if rank == 0:
        sv = leg["served"]
        line = {"metric": "served graphs/s", "value": world * sv["graphs_per_s"], "unit": "graphs/s",
                "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": sv["span_s"] * 1e3,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": leg["workload"], "requests": leg["requests"], "pool": leg["pool_graphs"],
                           "l2": "inputs larger than L2", "parallelism": "replicas" if world > 1 else "single"},
                "roofline": None, "cpu_baseline": None,
                "e2e": {"value": world * sv["graphs_per_s"], "unit": "graphs/s",
                        "h2d_bytes_per_step": 8 * leg["edges_in"], "d2h_bytes_per_step": 8 * leg["requests"]},
                "gpu_launches": sv["gpu_launches"], "clocks": clk, "serve": leg}
        print(json.dumps(line), flush=True)
    return 0


def surrogate_part_range(world, rank, nparts):
    """Receiving parts [lo, hi) of rank `rank` when `nparts` parts are shared by `world` ranks:
    contiguous ranges whose sizes differ by at most one."""
    return rank * nparts // world, (rank + 1) * nparts // world


def run_partitioned_surrogate(args, rank, world, local):
    """One graph's N+ lists, held in page-locked host memory by every rank, counted by all ranks
    over Sec. IV's non-overlapping partition: equal-work cuts (Sec. IV-F cost) into one part per
    rank, each rank counting the messages its part receives (tc_count_surrogate with its part
    range); one uint64 sum over the ranks gives T.  Strong scaling."""
    import torch
    import paper_1406_5687_gb300 as tc
    from graphgen import workloads as W
    torch.cuda.set_device(local)
    pg = init_replicas(world)
    spec = W.SINGLE[args.workload]
    s, d = spec.edges()
    s_dev, d_dev = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    del s, d
    stream = torch.cuda.current_stream()
    g0 = tc.Graph.build(s_dev, d_dev, spec.n)
    T_ref, m_hat = g0.count(stream), g0.info()["m_hat"]
    _, off, cols, _ = g0.csr()
    g0.free()
    del s_dev, d_dev
    off_h, cols_h = off.cpu().pin_memory(), cols.cpu().pin_memory()
    del off, cols
    torch.cuda.empty_cache()
    cuts = tc.surrogate_plan(off_h, cols_h, nparts=world, fn=tc.TC_FN_NEW)
    lo, hi = surrogate_part_range(world, rank, len(cuts) - 1)

    def step():
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        part, _tab = tc.count_surrogate(off_h, cols_h, cuts, part_lo=lo, part_hi=hi, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), part

    for _ in range(args.warmup):
        step()
    if pg:
        pg.barrier()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    l0 = tc.kernel_launches()
    steps = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    launches = tc.kernel_launches() - l0
    clk = clocks.stop()
    total_ms = max_over_ranks(pg, sum(x[0] for x in steps))
    T = sum_over_ranks(pg, steps[-1][1])
    if pg:
        pg.barrier()
    if T != T_ref:
        raise RuntimeError(f"partial counts sum to {T}, not {T_ref}")
    if rank == 0:
        line = {"metric": METRIC, "value": replica_throughput(1, args.steps, m_hat, total_ms), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT[args.workload], "m_hat": m_hat, "triangles": T,
                           "l2": "inputs larger than L2", "lists": "page-locked host memory",
                           "parallelism": f"non-overlapping partition, one equal-work part per rank, {world} ranks"},
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def run_partitioned(args, rank, world, local):
    """One graph counted by all ranks: each builds it (a replica) and counts part `rank` of
    `world` cost-balanced parts of its tasks (tc_count_partition); one uint64 sum over the ranks
    gives T.  The work is fixed as ranks are added: strong scaling."""
    import torch
    import paper_1406_5687_gb300 as tc
    from graphgen import workloads as W
    torch.cuda.set_device(local)
    pg = init_replicas(world)
    spec = W.SINGLE[args.workload]
    s, d = spec.edges()
    s_dev, d_dev = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    del s, d
    stream = torch.cuda.current_stream()
    opt = tc.default_options()
    g0 = tc.Graph.build(s_dev, d_dev, spec.n, opt)
    T_ref, m_hat = g0.count(stream), g0.info()["m_hat"]
    g0.free()

    def step():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        g = tc.Graph.build(s_dev, d_dev, spec.n, opt, stream=stream)
        e1.record(stream)
        part = g.count_partition(rank, world, stream)
        e2.record(stream)
        e2.synchronize()
        g.free()
        return e0.elapsed_time(e2), e0.elapsed_time(e1), e1.elapsed_time(e2), part

    for _ in range(args.warmup):
        step()
    if pg:
        pg.barrier()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    l0 = tc.kernel_launches()
    steps = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    launches = tc.kernel_launches() - l0
    clk = clocks.stop()
    total_ms = max_over_ranks(pg, sum(x[0] for x in steps))
    T = sum_over_ranks(pg, steps[-1][3])
    if pg:
        pg.barrier()
    if T != T_ref:
        raise RuntimeError(f"partial counts sum to {T}, not {T_ref}")
    if rank == 0:
        line = {"metric": METRIC, "value": replica_throughput(1, args.steps, m_hat, total_ms), "unit": UNIT,
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "int32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT[args.workload], "m_hat": m_hat, "triangles": T,
                           "l2": "inputs larger than L2", "parallelism": f"cost-partitioned over {world} ranks"},
                "phases_ms": {"build": statistics.mean(x[1] for x in steps),
                              "count_part": statistics.mean(x[2] for x in steps)},
                "roofline": None, "cpu_baseline": None, "e2e": None, "gpu_launches": launches, "clocks": clk}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


COST_MODELS = ["edge", "merge", "one", "degree", "patric", "new"]


def run_ablation(args, local):
    """Cost functions (Sec. IV-B, IV-F, V-A) and the static share of Eq. 1 on the GPU: the same
    built graph counted under each setting; per class, the kernel time and the spread of the
    workers' busy clocks (the idle time of Sec. V-E: max busy vs median busy)."""
    import numpy as np
    import torch
    import paper_1406_5687_gb300 as tc
    from graphgen import workloads as W
    torch.cuda.set_device(local)
    spec = W.SINGLE[args.workload]
    s, d = spec.edges()
    g = tc.Graph.build(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), spec.n)
    T_ref = g.count()
    for model in range(6):
        for sp in (0, 50, 100):
            opt = tc.default_options(cost_model=model, static_percent=sp)
            best = None
            for _ in range(max(2, args.steps)):
                T, meta, _, busy = g.count_ex(opt, busy=True)
                if T != T_ref:
                    raise RuntimeError("the count changed with the cost model")
                if best is None or meta["kernel_ms"] < best[0]["kernel_ms"]:
                    best = (meta, busy.cpu().numpy())
            meta, b = best
            ws = meta["n_workers"][0]
            row = {"workload": WORKLOAD_TEXT[args.workload], "cost_model": COST_MODELS[model], "static_percent": sp,
                   "kernel_small_ms": meta["kernel_small_ms"], "kernel_big_ms": meta["kernel_big_ms"],
                   "prefix_ms": meta["prefix_ms"], "chunks": [int(meta["min_chunk"][0]), int(meta["min_chunk"][1])]}
            for cls, part in (("small", b[:ws]), ("big", b[ws:])):
                cyc = part[:, 0].astype(np.float64)
                if len(cyc) and cyc.max() > 0:
                    row[f"{cls}_busy_max_over_median"] = float(cyc.max() / max(np.median(cyc), 1.0))
                    row[f"{cls}_idle_fraction"] = float(1.0 - cyc.mean() / cyc.max())
                    row[f"{cls}_chunks_per_worker"] = float(part[:, 1].mean())
            print(json.dumps(row), flush=True)
    g.free()
    return 0


def run_gpu(args, rank, world, local):
    import numpy as np
    import torch
    import paper_1406_5687_gb300 as tc
    from graphgen import workloads as W

    if args.ablation:
        return run_ablation(args, local) if rank == 0 else 0
    if args.partitioned:
        if args.partition_mode == "surrogate":
            return run_partitioned_surrogate(args, rank, world, local)
        return run_partitioned(args, rank, world, local)

    if args.workload == "batch":
        return run_batch_only(args, rank, world, local)
    if args.workload == "serve":
        return run_serve_only(args, rank, world, local)
    torch.cuda.set_device(local)
    pg = init_replicas(world)
    spec = W.SINGLE[args.workload]
    s, d = spec.edges()
    m_in = len(s)
    s_pin = torch.from_numpy(s).pin_memory()
    d_pin = torch.from_numpy(d).pin_memory()
    del s, d
    s_dev, d_dev = s_pin.cuda(), d_pin.cuda()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    opt = tc.default_options()
    g = tc.Graph.build(s_dev, d_dev, spec.n, opt)
    info = g.info()
    T_ref = g.count()
    alg = algorithmic_bytes(g, opt)
    g.free()
    m_hat = info["m_hat"]

    def device_step():
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        gg = tc.Graph.build(s_dev, d_dev, spec.n, opt)
        e1.record(stream)
        T, meta, _, _ = gg.count_ex(timing=True)
        e2.record(stream)
        e2.synchronize()
        gg.free()
        if T != T_ref:
            raise RuntimeError(f"count changed between steps: {T} != {T_ref}")
        return (e0.elapsed_time(e2), e0.elapsed_time(e1), e1.elapsed_time(e2), meta["kernel_ms"], meta["prefix_ms"],
                meta["kernel_small_ms"], meta["kernel_big_ms"])

    for _ in range(args.warmup):
        device_step()
    torch.cuda.synchronize()
    if pg:
        pg.barrier()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    clocks = ClockSampler(gpu_index)
    clocks.start()
    l0 = tc.kernel_launches()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    steps = [device_step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    launches = tc.kernel_launches() - l0
    clk = clocks.stop()
    total_ms = max_over_ranks(pg, sum(x[0] for x in steps))
    if pg:
        pg.barrier()
    value = replica_throughput(world, args.steps, m_hat, total_ms)
    build_ms = statistics.mean(x[1] for x in steps)
    count_ms = statistics.mean(x[2] for x in steps)
    kernel_ms = statistics.mean(x[3] for x in steps)
    prefix_ms = statistics.mean(x[4] for x in steps)
    small_ms = statistics.mean(x[5] for x in steps)
    big_ms = statistics.mean(x[6] for x in steps)

    # e2e: edge list in pinned host memory, copies and the 8-byte result read inside the step
    e2e = None
    if not args.no_e2e:
        def host_step():
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gg = tc.Graph.build(s_pin, d_pin, spec.n, opt)
            T = gg.count()
            e1.record(stream)
            e1.synchronize()
            gg.free()
            if T != T_ref:
                raise RuntimeError("count changed in the e2e run")
            return e0.elapsed_time(e1)
        host_step()
        e2e_ms = max_over_ranks(pg, sum(host_step() for _ in range(args.steps)))
        e2e = {"value": replica_throughput(world, args.steps, m_hat, e2e_ms), "unit": UNIT,
               "h2d_bytes_per_step": 8 * m_in, "d2h_bytes_per_step": 8,
               "ms_per_step": e2e_ms / args.steps}

    # the optional outputs of the same count (outside the timed region): per-vertex T_v,
    # per-edge counts and clustering coefficients, CUDA events on the same stream
    extras = None
    if rank == 0 and not args.no_per_vertex:
        gg = tc.Graph.build(s_dev, d_dev, spec.n, opt)
        def timed(f):
            best = None
            for _ in range(2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r = f()
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None or ms < best else best
            return best, r
        count_ms1, _ = timed(lambda: gg.count(stream))
        pv_ms, (T_pv, tv) = timed(lambda: gg.count_per_vertex(stream))
        pe_ms, (T_pe, _pe) = timed(lambda: gg.count_per_edge(stream))
        cc_ms, _cc = timed(lambda: gg.clustering(tv, stream))
        if T_pv != T_ref or T_pe != T_ref or int(tv.sum().item()) != 3 * T_ref:
            raise RuntimeError("per-vertex or per-edge count disagrees with the total")
        extras = {"count_ms": count_ms1, "per_vertex_ms": pv_ms, "per_edge_ms": pe_ms, "clustering_ms": cc_ms,
                  "note": "tc_count, tc_count_per_vertex (T_v), tc_count_per_edge and tc_clustering on the same built "
                          "graph, each the faster of two runs"}
        del tv, _pe, _cc
        gg.free()

    surrogate = None
    if rank == 0 and not args.no_surrogate:
        surrogate = surrogate_leg(s_dev, d_dev, spec.n, opt, T_ref, stream, fraction=args.surrogate_fraction)

    peak, peak_kind = measured_peaks()
    # The roofline is that of the dominant kernel, k_count_big (the big class of step a7-a8):
    # its algorithmic bytes over its own average duration, timed with CUDA events on the
    # stream it runs on.
    achieved = alg["big"]["bytes"] / (big_ms / 1e3) / 1e9
    roofline = {"kernel": "k_count_big (big-owner class of the intersection, steps a7-a8)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": f"hbm_gbs of {peak_kind}", "traffic": stored_traffic(args.workload),
                "algorithmic_bytes": alg["big"]["bytes"], "launch_ms": big_ms,
                "both_count_kernels": {"algorithmic_bytes": alg["total"], "ms": kernel_ms,
                                       "gbs": alg["total"] / (kernel_ms / 1e3) / 1e9,
                                       "frac": alg["total"] / (kernel_ms / 1e3) / 1e9 / peak},
                "merge_model": {"bytes": alg["merge"], "gbs": alg["merge"] / (kernel_ms / 1e3) / 1e9,
                                "note": "4 (sum over oriented edges of |N+(u)| + m_hat) + 16 n per count, "
                                        "over both count kernels"}}

    bb = build_bytes(dict(info, m_input=m_in))
    build_roofline = {"phase": "build (a1-a5 and the task array)", "bound": "hbm", "bytes": bb["bytes"],
                      "ms": build_ms, "achieved": bb["bytes"] / (build_ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                      "frac": bb["bytes"] / (build_ms / 1e3) / 1e9 / peak, "peak_source": f"hbm_gbs of {peak_kind}",
                      "sort_passes": bb["sort_passes"], "sort_bytes": bb["sort_bytes"], "terms": bb["terms"]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload, CPU_SAMPLE_PAIRS[args.workload])
        cpu["gpu_same_graph"] = {"step_ms": total_ms / args.steps, "build_ms": build_ms, "count_ms": count_ms}

    batch = None
    if rank == 0 and not args.no_batch:
        batch = batch_leg(args.batch_graphs or 4096, 2, 1, pack_edges=args.pack_edges)
    serve = None
    if rank == 0 and not args.no_serve:
        serve = serve_leg(args.serve_requests or 2000, args.serve_pool or 256, args.serve_slots, args.serve_group_edges)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": WORKLOAD_TEXT[args.workload], "m_input": m_in, "m_hat": m_hat,
                           "n": info["n"], "triangles": T_ref, "tasks": info["tasks"],
                           "max_degree": info["max_degree"], "max_dhat": info["max_dhat"],
                           "l2": "inputs larger than L2 (edge list, lists and tasks each exceed 129 MB)",
                           "parallelism": "replicas" if world > 1 else "single",
                           "options": {"piece": opt.piece, "warps_per_block": opt.warps_per_block,
                                       "big_warps": opt.big_warps, "small_max": opt.small_max,
                                       "cost_model": "edge", "static_percent": opt.static_percent}},
                "phases_ms": {"build": build_ms, "count": count_ms, "count_prefix": prefix_ms,
                              "count_kernels": kernel_ms, "count_kernel_small": small_ms, "count_kernel_big": big_ms},
                "count_only": {"value": m_hat / (count_ms / 1e3), "unit": UNIT,
                               "note": "m_hat / (cost prefix + schedule + intersection), lists resident"},
                "roofline": roofline, "build_roofline": build_roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches,
                "clocks": clk, "work": {"small": alg["small"], "big": alg["big"]}, "wall_s_timed": t_wall,
                "per_vertex": extras, "surrogate": surrogate, "batch": batch, "serve": serve}
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def main():
    args = parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_gpu(args, rank, world, local)


if __name__ == "__main__":
    sys.exit(main())
