"""Plan-time validation of the lowered descriptors, fuzzed on the CPU.

Every plan is lowered and then checked on the host before anything can be
launched: every leaf, operand and output range lies inside its arena (both
schedules and the 8-bit-prime layout with its doubled fp16-plane extents),
each step's bit maps cover the operands' free bits exactly once, and no
output of a tree level overlaps anything the level reads or writes.  A
failed check is an "internal:" TNC_ERR_INVALID.  These tests drive that check
with random formulas of every clause kind (open variables, empty clauses,
variables in no clause), every planner and random explicit orders, and tie
the plans to the oracle: contracting along a plan's own order gives the
oracle's count (Sec. 2.1: the count does not depend on the order).
"""
import random

import pytest

import oracle

from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import tnc
from _util import random_formula, random_order

HEURISTICS = ("greedy", "bisect", "gn", "best", "portfolio", "coarsen")


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


def _plan_or_too_large(net, **kw):
    """A plan, or None where the order exceeds the rank cap (TNC_ERR_TOO_LARGE
    is the documented refusal); any other error fails the test."""
    try:
        return tnc.plan(net, **kw)
    except tnc.TncError as e:
        assert e.code == -2, str(e)
        return None


def test_random_formulas_lower_and_validate_under_every_planner():
    rng = random.Random(1805)
    planned = 0
    for i in range(160):
        n = rng.randint(1, 26)
        f = random_formula(rng, n, rng.randint(0, 34), n_open=rng.randint(0, min(3, n)),
                           allow_empty=True)
        try:
            net = tnc.build_network(f)
        except tnc.TncError as e:  # a variable in more than 32 clauses is refused
            assert e.code == -2, str(e)
            continue
        L = f.n_vars + f.n_cons
        for h in HEURISTICS:
            p = _plan_or_too_large(net, heuristic=h, rank_cap=40, seed=i)
            if p is None:
                continue
            planned += 1
            assert p.stats.n_steps == max(L - 1, 0)
            assert p.stats.n_leaves == L
            steps = p.steps()
            assert len(steps) == p.stats.n_steps
        for _ in range(2):
            p = _plan_or_too_large(net, order=random_order(rng, f), rank_cap=40)
            if p is not None:
                planned += 1
                assert p.stats.n_steps == max(L - 1, 0)
    assert planned >= 120 * len(HEURISTICS)


def test_batched_planning_validates_like_single_planning():
    """tnc_plan_many (OpenMP over formulas) lowers and validates every plan as
    tnc_plan does; the costs agree formula by formula."""
    rng = random.Random(7)
    forms = [random_formula(rng, rng.randint(2, 20), rng.randint(1, 24), n_open=rng.randint(0, 2))
             for _ in range(64)]
    for h in ("bisect", "coarsen"):
        many = tnc.plan_many(forms, heuristic=h, rank_cap=64)
        for f, p in zip(forms, many):
            one = tnc.plan(tnc.build_network(f), heuristic=h, rank_cap=64)
            assert (p.stats.max_rank, p.stats.total_macs, p.stats.total_entries) == \
                (one.stats.max_rank, one.stats.total_macs, one.stats.total_entries)


@pytest.mark.parametrize("seed", range(4))
def test_library_plans_give_the_oracle_count_along_their_order(seed):
    """The oracle contracting along each library plan's order (an explicit
    pairwise order) gets the count of its own default order."""
    rng = random.Random(100 + seed)
    f = random_formula(rng, 12, 14, n_open=rng.randint(0, 2), weights=(0, 1, 3, 7))
    want = oracle.count(f, max_rank=26)
    net = tnc.build_network(f)
    for h in HEURISTICS:
        p = tnc.plan(net, heuristic=h, rank_cap=26)
        assert oracle.count(f, order=p.steps(), max_rank=26) == want, h
