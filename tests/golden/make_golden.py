"""Write the stored expected values under tests/golden/ by calling only the oracle.

    python tests/golden/make_golden.py

er_10k.txt: the Erdos-Renyi G(n=10,000, m=100,000) graph of seed 0 (integer-only
generator, so identical on every platform) counted by the oracle (Fig. 1).
"""
import hashlib
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from graphgen import workloads as W  # noqa: E402


def main():
    spec = W.ER_10K
    s, d = spec.edges()
    g = oracle.simple_graph(spec.n, s, d)
    csr = oracle.oriented_csr(g)
    T, per_edge, tv = oracle.count(csr, per_edge=True, per_vertex=True)
    lines = [
        "# Erdos-Renyi G(n=10000, m=100000), seed 0; values written by make_golden.py from the oracle (Fig. 1)",
        f"n {spec.n}",
        f"m_in {len(s)}",
        f"m_hat {g.m_hat}",
        f"triangles {T}",
        f"max_degree {int(csr.deg.max())}",
        f"max_dhat {int(np.diff(csr.off).max())}",
        f"sum_t_v {int(tv.sum())}",
        f"sha256_t_v {hashlib.sha256(tv.astype('<u8').tobytes()).hexdigest()}",
        f"sha256_per_edge {hashlib.sha256(per_edge.astype('<u4').tobytes()).hexdigest()}",
        f"sha256_cols {hashlib.sha256(csr.cols.astype('<i4').tobytes()).hexdigest()}",
    ]
    with open(os.path.join(HERE, "er_10k.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")
    print("\n".join(lines))


if __name__ == "__main__":
    main()
