"""The stored exact counts of tests/golden/dense_branch_counts.json are the
oracle's: the cheapest case is recomputed here by the oracle, and every stored
count lies between bounds that hold for any connected cubic graph other than
K4 (#VC = #IS; by Brooks' theorem such a graph is 3-colourable, so it has an
independent set of at least n/3 vertices, all of whose subsets are
independent: #IS >= 2^(n/3); and not every subset is a cover: #VC < 2^n)."""
import json
import os

import oracle
from paper_1805_00475_gb300 import instances as I

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dense_branch_counts.json")


def test_golden_dense_counts_are_the_oracles():
    with open(GOLDEN) as fh:
        cases = json.load(fh)["cases"]
    c = min(cases, key=lambda x: x["n"])
    assert oracle.count(I.cubic_vertex_cover(c["n"], c["seed"]), max_rank=26) == [int(c["count"])]
    for c in cases:
        n, v = c["n"], int(c["count"])
        assert 2 ** (n / 3) <= v < 2 ** n
