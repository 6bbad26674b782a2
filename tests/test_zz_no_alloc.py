"""tnc_contract_noalloc: the entry point for callers that cannot allocate
device memory (their device memory belongs to another allocator, or they
cannot afford cudaMalloc/cudaFree in their loop).  Its scratch is a fixed
array inside libtnc, so the call allocates nothing on the device.

Each case calls it twice in a row through the C ABI and compares both results
with tnc_contract (which uses a caller-allocated workspace) and with the CPU
oracle's exact counts, bit for bit: the counts are exact integers, so the
tolerance is zero.  The second call runs on whatever the first left in the
shared array.  This file is collected last so
that a run stopping at the first failure has run every other test before it;
it also passes alone in a fresh process.
"""
import random
import time

import pytest

import oracle

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


def _exact(a: tnc.Count, f):
    """Every residue and every CRT value against the oracle's exact counts."""
    want = oracle.count(f, max_rank=26)
    assert a.residues.tolist() == oracle.residues(want, a.primes)
    if a.flags == 0:  # certified: the CRT value is the count itself
        assert a.counts == want
    else:  # the count may exceed the product of the primes: its residue class
        m = 1
        for q in a.primes:
            m *= q
        assert a.counts == [w % m for w in want]


CASES = [
    ("worked_example", I.worked_example(), 2, "gn"),
    ("one_in_three_n20", I.one_in_three(20, 12, 3), 1, "bisect"),
    ("cubic_vc_n60", I.cubic_vertex_cover(60, 4), 4, "gn"),
    # the last step is a dot product over 2^16 shared values (no output bits):
    # split over K into blocks
    ("cubic_vc_n90_dot_2^16", I.cubic_vertex_cover(90, 4), 4, "bisect"),
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
    _exact(first, f)
    _exact(second, f)


def test_noalloc_worked_example_and_k4_hand_counts():
    """Values fixed by the paper and by hand: the worked example's open
    network gives [[3, 3], [3, 4]] (Sec. 2.1); K4 has 5 vertex covers."""
    r = tnc.contract_noalloc(tnc.plan_formula(I.worked_example(), heuristic="gn"), n_residues=2)
    assert r.counts == [3, 3, 3, 4]
    r = tnc.contract_noalloc(tnc.plan_formula(I.vertex_cover_formula(4, I.complete_graph(4))), n_residues=1)
    assert r.counts == [5]


def test_noalloc_splits_long_dot_products():
    """A final dot product of two rank-18 tensors runs as split-K blocks (as in
    tnc_contract), not on a single thread: launch record and time."""
    import torch
    f = I.cubic_vertex_cover(100, 7)
    p = tnc.plan_formula(f, heuristic="bisect", rank_cap=24)
    ref = tnc.contract(p, n_residues=4)
    assert tnc.contract_noalloc(p, n_residues=4).counts == ref.counts
    assert tnc.last_launch_counts()["splitk"] >= 1

    def timed(fn, reps=5):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        return (time.perf_counter() - t) / reps

    t_ref = timed(lambda: tnc.contract(p, n_residues=4))
    t_na = timed(lambda: tnc.contract_noalloc(p, n_residues=4))
    assert t_na < 4 * t_ref + 0.02, (t_na, t_ref)


def test_noalloc_rejects_tensor_core_paths():
    p = tnc.plan_formula(I.cubic_vertex_cover(20, 0))
    for path in ("tc", "tc_p8"):
        with pytest.raises(tnc.TncError) as e:
            tnc.contract_noalloc(p, n_residues=2, path=path)
        assert e.value.code == -1 and "TNC_PATH_INT64 only" in str(e.value)


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
