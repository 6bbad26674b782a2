"""Every branch of the two tensor-core step kernels against the CPU oracle.

The formulas (#Cubic-Vertex-Cover on 100..130 vertices) have tensor-greedy
plans of rank <= 24 whose dense steps, between them, take every branch of
the dense kernels: 256-wide tiles on the 8-bit-prime path (two residues per
TMEM round; 256 x 256 tiles on CTA pairs sharing one MMA), several 1024-value chunks reduced mod p in TMEM before the next
accumulates on top, K splits on both tensor-core paths, operands read
K-contiguous and row-contiguous, and dense outputs written straight to the
fp16 planes of the next dense step.  The exact counts come
from tests/golden/dense_branch_counts.json, written by the oracle alone
(tests/golden/make_dense_counts.py).  Which branches ran is read from the
library's own launch record (tnc_last_launch_counts), not from a restatement
of its dispatch rule.  Residues are compared one by one with the exact count
mod each prime, and the CRT value with the count.
"""
import json
import math
import os

import pytest

from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "dense_branch_counts.json")
with open(GOLDEN) as fh:
    CASES = [(c["n"], c["seed"], int(c["count"])) for c in json.load(fh)["cases"]]
PATHS = ("int64", "tc", "tc_p8")


def _n_residues(path, log2_bound):
    """Enough primes that their product exceeds the certified bound."""
    primes = tnc.default_primes(53 if path == "tc_p8" else 16, path)
    bits, n = 0.0, 0
    while bits <= log2_bound + 1:
        bits += math.log2(primes[n])
        n += 1
    return n


@pytest.fixture(scope="module")
def runs():
    tnc_build.build()
    out = {}
    for n, seed, exact in CASES:
        p = tnc.plan_formula(I.cubic_vertex_cover(n, seed), heuristic="greedy", rank_cap=26)
        for path in PATHS:
            r = tnc.contract(p, n_residues=_n_residues(path, p.stats.log2_bound), path=path)
            out[(n, seed, path)] = (r, tnc.last_launch_counts(), exact)
    return out


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,seed", [(c[0], c[1]) for c in CASES])
def test_dense_branches_match_oracle(runs, n, seed, path):
    r, lc, exact = runs[(n, seed, path)]
    assert r.flags == 0
    assert [int(x) for x in r.residues[0]] == [exact % q for q in r.primes]
    assert r.counts == [exact]
    if path == "tc":
        assert lc["tc_gemm"] >= 1 and lc["p8_gemm"] == 0
    elif path == "tc_p8":
        assert lc["p8_gemm"] >= 1 and lc["tc_gemm"] == 0
        # a step packs unless both operands came as fp16 planes from dense steps
        assert lc["p8_pack"] <= lc["p8_gemm"] and lc["p8_pack"] >= lc["p8_gemm"] - lc["p8_direct_in"]
        assert lc["p8_direct_in"] == lc["p8_direct_out"] <= lc["p8_mn"] <= 2 * lc["p8_gemm"]
    else:
        assert lc["tc_gemm"] == 0 and lc["p8_gemm"] == 0


def test_dense_cases_take_every_branch(runs):
    """The launch records of the cases above, together, show every branch."""
    tc = [lc for (n, s, path), (_, lc, _) in runs.items() if path == "tc"]
    p8 = [lc for (n, s, path), (_, lc, _) in runs.items() if path == "tc_p8"]
    for w in (64, 128, 256):
        assert sum(lc["p8_tile_n"][w] for lc in p8) >= 1, f"no {w}-wide p8 tile"
    assert sum(lc["p8_cta_pair"] for lc in p8) >= 1, "no 256 x 256 tile on a CTA pair"
    assert all(lc["p8_cta_pair"] <= lc["p8_tile_n"][256] for lc in p8)
    assert max(lc["p8_max_chunks"] for lc in p8) >= 2, "no step reduced in TMEM between chunks"
    assert sum(lc["p8_split"] for lc in p8) >= 1, "no p8 K split"
    assert sum(lc["tc_split"] for lc in tc) >= 1, "no limb-path K split"
    assert sum(lc["tc_gemm"] - lc["tc_split"] for lc in tc) >= 1, "no unsplit limb-path step"
    assert sum(lc["p8_gemm"] - lc["p8_split"] for lc in p8) >= 1, "no unsplit p8 step"
    assert sum(lc["p8_direct_out"] for lc in p8) >= 1, "no dense step wrote its consumer's fp16 planes"
    assert sum(lc["p8_mn"] - lc["p8_direct_in"] for lc in p8) >= 1, "no row-contiguous operand packed"
    assert sum(2 * lc["p8_gemm"] - lc["p8_mn"] for lc in p8) >= 1, "no K-contiguous operand"
    assert sum(lc["p8_pairs"] for lc in p8) >= 1, "no epilogue writing pairs of entries"
    assert sum(lc["p8_gemm"] - lc["p8_pairs"] for lc in p8) >= 1, "no epilogue writing single entries"
    # one formula alone reaches all four
    both = [(n, s) for (n, s, path), (_, lc, _) in runs.items() if path == "tc_p8" and lc["p8_tile_n"][256]
            and lc["p8_max_chunks"] >= 2 and lc["p8_split"] and runs[(n, s, "tc")][1]["tc_split"]]
    assert both
