"""Writes tests/golden/dense_branch_counts.json: exact counts of the
#Cubic-Vertex-Cover formulas whose tensor-greedy plans reach every branch of
the two tensor-core step kernels (256-wide tiles, several 1024-value chunks
reduced in TMEM, K splits on both dense paths), computed by the CPU oracle
alone (pairwise big-integer contraction of the paper's network, Sec. 2.1,
along the oracle's own tensor-greedy order, Sec. 3.1.1).

    python tests/golden/make_dense_counts.py

Only oracle/ and the seeded instance generators are used: no value here comes
from the library under test.  The oracle is pinned by tests/test_oracle_pins.py.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1805_00475_gb300 import instances as I  # noqa: E402

# (vertices, seed): random simple connected cubic graphs (configuration model
# with rejection); the count is the number of vertex covers (Eq. or on every
# edge, Eq. var on every vertex).
CASES = [(100, 11), (110, 6), (110, 8), (110, 9), (130, 6)]


def main():
    out = {"what": "number of vertex covers of I.cubic_vertex_cover(n, seed)",
           "how": "oracle.contract (C big integers, tensor-greedy order, max rank 26)",
           "cite": "Sec. 2.1 (network and full trace), Sec. 3.1.1 (tensor-greedy)",
           "cases": []}
    for n, seed in CASES:
        t = time.time()
        counts, max_rank, _ = oracle.contract(I.cubic_vertex_cover(n, seed), max_rank=26)
        out["cases"].append({"n": n, "seed": seed, "count": str(counts[0]), "oracle_max_rank": max_rank})
        print(n, seed, counts[0], f"{time.time() - t:.1f} s", flush=True)
    with open(os.path.join(HERE, "dense_branch_counts.json"), "w") as fh:
        json.dump(out, fh, indent=1)
        fh.write("\n")


if __name__ == "__main__":
    main()
