"""tnc_contract_noalloc: the entry point for callers that cannot allocate
device memory (their device memory belongs to another allocator, or they
cannot afford cudaMalloc/cudaFree in their loop).  Its scratch is a fixed
array inside libtnc, so the call allocates nothing on the device.

Each case calls it twice in a row through the C ABI and compares both results
with tnc_contract (which uses a caller-allocated workspace) bit for bit: the
counts are exact integers, so the tolerance is zero.  The second call runs on
whatever the first left in the shared array.  This file is collected last so
that a run stopping at the first failure has run every other test before it;
it also passes alone in a fresh process.
"""
import random

import pytest

from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc
from _util import random_formula

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


def _same(a: tnc.Count, b: tnc.Count):
    assert a.counts == b.counts
    assert a.residues.tolist() == b.residues.tolist()
    assert a.primes == b.primes and a.flags == b.flags


CASES = [
    ("worked_example", I.worked_example(), 2, "gn"),
    ("one_in_three_n20", I.one_in_three(20, 12, 3), 1, "bisect"),
    ("cubic_vc_n60", I.cubic_vertex_cover(60, 4), 4, "gn"),
    ("lucas_cycle_130", I.vertex_cover_formula(130, I.cycle_graph(130)), 8, "bisect"),
    ("weighted_open", random_formula(random.Random(11), 12, 10, 3, weights=(0, 1, 3, 2 ** 32 - 1)), 5, "greedy"),
    ("empty", I.Formula(0, [], []), 3, "greedy"),
]


@pytest.mark.parametrize("name,f,R,h", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_contract_twice(name, f, R, h):
    import torch
    p = tnc.plan_formula(f, heuristic=h)
    ref = tnc.contract(p, n_residues=R)
    stream = torch.cuda.Stream()
    first = tnc.contract_noalloc(p, n_residues=R, stream=stream)
    second = tnc.contract_noalloc(p, n_residues=R, stream=stream)
    _same(first, ref)
    _same(second, ref)


def test_noalloc_alternating_plans_reuse_the_array():
    """A small plan after a larger one must not see the larger one's leftovers."""
    big = tnc.plan_formula(I.cubic_vertex_cover(60, 7), heuristic="gn")
    small = tnc.plan_formula(I.one_in_three(20, 12, 1), heuristic="greedy")
    want_big, want_small = tnc.contract(big, n_residues=4), tnc.contract(small, n_residues=4)
    for _ in range(2):
        _same(tnc.contract_noalloc(big, n_residues=4), want_big)
        _same(tnc.contract_noalloc(small, n_residues=4), want_small)


def test_noalloc_rejects_plans_beyond_the_array():
    p = tnc.plan_formula(I.cubic_vertex_cover(180, 0), heuristic="gn")
    assert tnc.workspace_bytes(p, 8) > tnc.NOALLOC_SCRATCH_BYTES
    with pytest.raises(tnc.TncError) as e:
        tnc.contract_noalloc(p, n_residues=8)
    assert e.value.code == -2 and "scratch" in str(e.value)
