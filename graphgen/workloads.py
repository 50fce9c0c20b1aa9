"""Named synthetic workloads.

The paper measures on web-BerkStan, LiveJournal, Miami, Twitter and PA(n,d)
graphs (Sec. II, Table I); none of those datasets is available here, so these
seeded synthetic graphs stand in for them: Barabasi-Albert for the paper's
preferential-attachment PA(n,d) family at d = 100 (as in PA(10M,100) of
Table II), and Chung-Lu with exponent 2.1 for its skewed web and social graphs.

=====  =====================================================================
name   recipe
=====  =====================================================================
er     Erdos-Renyi G(n=10,000, m=100,000), seed 0
ba     Barabasi-Albert n=1,000,000, k=50 (avg degree 100), seed 1
cl     Chung-Lu n=10,000,000, exponent 2.1, mean weight 40, w_0 = 1e5,
       2.0e8 edge draws (self-loops dropped and repeats merged by the counter's
       input policy), seed 2
cl_twitter  the same recipe at Twitter's size (Table I): n=41,650,000,
       mean weight 115, w_0 = 3e6, 2.4e9 edge draws, seed 5
batch  4096 graphs, seed 3: even index Erdos-Renyi, odd index Barabasi-Albert;
       n log-uniform in [1e3, 2e5]; average degree uniform in [8, 128]
serve  Poisson arrivals at 2,000 graphs/s of Chung-Lu graphs: exponent uniform
       in [2.1, 2.8], n log-uniform in [1e4, 2e6], average degree uniform in
       [16, 96], w_0 = min(n/2, 5 sqrt(n d)); seed 4
=====  =====================================================================
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import barabasi_albert, chung_lu, draw, erdos_renyi


@dataclass(frozen=True)
class GraphSpec:
    family: str          # "er" | "ba" | "cl"
    n: int
    seed: int
    m: int = 0           # er: edge count
    k: int = 0           # ba: edges per new vertex
    gamma: float = 0.0   # cl
    avg_deg: float = 0.0  # cl
    w_max: float = 0.0   # cl
    draws: int = 0       # cl

    def edges(self):
        """Generate (src, dst) int32 arrays for this spec."""
        if self.family == "er":
            return erdos_renyi(self.n, self.m, self.seed)
        if self.family == "ba":
            return barabasi_albert(self.n, self.k, self.seed)
        if self.family == "cl":
            return chung_lu(self.n, self.gamma, self.avg_deg, self.w_max, self.draws, self.seed)
        raise ValueError(self.family)

    @property
    def num_input_edges(self) -> int:
        if self.family == "er":
            return self.m
        if self.family == "ba":
            return self.k * (self.n - self.k)
        return self.draws


ER_10K = GraphSpec("er", n=10_000, m=100_000, seed=0)
BA_1M = GraphSpec("ba", n=1_000_000, k=50, seed=1)
CL_10M = GraphSpec("cl", n=10_000_000, gamma=2.1, avg_deg=40.0, w_max=1e5, draws=200_000_000, seed=2)

# the Chung-Lu recipe at one fifth of the vertices and edges (w_0 scaled by sqrt(n)), for
# profiling captures that must hold only a few GB on the device
CL_2M = GraphSpec("cl", n=2_000_000, gamma=2.1, avg_deg=40.0, w_max=44721.0, draws=40_000_000, seed=2)

# the Chung-Lu recipe at the size of the paper's largest real graph (Twitter, Table I: 42M
# vertices, 2.4B edges): 41.65M vertices, 2.4e9 edge draws, mean weight 115, w_0 = 3e6
CL_TWITTER = GraphSpec("cl", n=41_650_000, gamma=2.1, avg_deg=115.0, w_max=3e6, draws=2_400_000_000, seed=5)

SINGLE = {"er": ER_10K, "ba": BA_1M, "cl": CL_10M, "cl_small": CL_2M, "cl_twitter": CL_TWITTER}


def _unit(seed: int, tag: int, i: int) -> float:
    """Uniform double in [0, 1) from draw i of stream (seed, tag)."""
    return (draw(seed, tag, i) >> 11) * (1.0 / 9007199254740992.0)


def batch_spec(j: int, seed: int = 3, n_lo: float = 1e3, n_hi: float = 2e5,
               d_lo: float = 8.0, d_hi: float = 128.0) -> GraphSpec:
    """Graph j of the batched workload (even j: Erdos-Renyi, odd j: Barabasi-Albert)."""
    u_n, u_d = _unit(seed, 10, 2 * j), _unit(seed, 10, 2 * j + 1)
    n = int(round(math.exp(math.log(n_lo) + u_n * (math.log(n_hi) - math.log(n_lo)))))
    d = d_lo + u_d * (d_hi - d_lo)
    gseed = int(draw(seed, 11, j))
    if j % 2 == 0:
        m = min(int(round(n * d / 2)), n * (n - 1) // 2)
        return GraphSpec("er", n=n, m=m, seed=gseed)
    k = max(1, int(round(d / 2)))
    return GraphSpec("ba", n=n, k=k, seed=gseed)


def batch_specs(count: int = 4096, seed: int = 3, **kw):
    return [batch_spec(j, seed, **kw) for j in range(count)]


def serve_spec(j: int, seed: int = 4, n_lo: float = 1e4, n_hi: float = 2e6,
               d_lo: float = 16.0, d_hi: float = 96.0) -> GraphSpec:
    """Graph j of the serving pool (Chung-Lu)."""
    u_g, u_n, u_d = (_unit(seed, 20, 3 * j + q) for q in range(3))
    gamma = 2.1 + 0.7 * u_g
    n = int(round(math.exp(math.log(n_lo) + u_n * (math.log(n_hi) - math.log(n_lo)))))
    d = d_lo + u_d * (d_hi - d_lo)
    w_max = min(n / 2.0, 5.0 * math.sqrt(n * d))
    draws = int(round(n * d / 2))
    return GraphSpec("cl", n=n, gamma=gamma, avg_deg=d, w_max=w_max, draws=draws, seed=int(draw(seed, 21, j)))


def poisson_arrivals(count: int, rate: float, seed: int = 4) -> np.ndarray:
    """Arrival times (seconds) of `count` requests of a Poisson process of the given rate."""
    gaps = np.array([-math.log(1.0 - _unit(seed, 22, i)) / rate for i in range(count)])
    return np.cumsum(gaps)
