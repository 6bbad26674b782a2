"""Bond slicing (host side): the count of a formula is the sum of the counts
of its slices (the oracle on every slice against the oracle on the whole),
open variables stay open, and the choice of sliced variables lowers the plan
rank of a large network."""
import itertools
import random

import pytest

import oracle
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import slicing as S
from paper_1805_00475_gb300 import tnc
from _util import random_formula


def _sum_of_slices(f, vs):
    total = None
    for bits in itertools.product((0, 1), repeat=len(vs)):
        c = oracle.count(S.slice_formula(f, dict(zip(vs, bits))))
        total = c if total is None else [a + b for a, b in zip(total, c)]
    return total


@pytest.mark.parametrize("seed", range(4))
def test_slices_sum_to_the_count(seed):
    for f in (I.one_in_three(18, 12, seed), I.cubic_vertex_cover(16, seed), I.random_k_cnf(16, 14, 3, seed),
              I.independent_set_formula(14, I.random_cubic_graph(14, seed)),
              random_formula(random.Random(seed), 14, 12, n_open=1)):
        whole = oracle.count(f)
        for vs in ([0], [1, 5], [2, 3, 7]):
            vs = [v for v in vs if v not in f.open_vars]
            assert _sum_of_slices(f, vs) == whole


def test_open_variables_stay_open():
    f = I.one_in_three(16, 10, 3)
    f.open_vars = [0, 4]
    assert _sum_of_slices(f, [2, 9]) == oracle.count(f)
    with pytest.raises(ValueError):
        S.slice_formula(f, {4: 1})


def test_fixed_variables_leave_the_network():
    f = I.cubic_vertex_cover(20, 1)
    g = S.slice_formula(f, {0: 1, 7: 0})
    assert g.n_vars == f.n_vars - 2
    assert all(k == I.KIND_TABLE for c, k in zip(g.clauses, g.kinds) if len(c) < 2)
    assert sum(len(c) for c in g.clauses) == sum(len(c) for c in f.clauses) - 6  # 3 bonds per cubic vertex


def test_slicing_lowers_the_rank_of_a_large_network():
    f = I.cubic_vertex_cover(180, 3)
    full = tnc.plan_formula(f, heuristic="best", rank_cap=40)
    vs = S.choose_slice_vars(f, 3)
    plans, forms = S.sliced_plans(f, vs)
    assert len(plans) == 8 and len(set(vs)) == 3
    assert max(p.stats.max_rank for p in plans) <= full.stats.max_rank - 2
    assert max(p.stats.arena_entries for p in plans) * 4 <= full.stats.arena_entries


def test_random_planar_cubic_graphs():
    """The planar generator: simple, cubic, connected, planar (networkx's
    planarity test), seeded; and the planner finds far lower max ranks on
    them than on unrestricted cubic graphs of the same size (the trend of the
    paper's Fig. 4c)."""
    nx = pytest.importorskip("networkx")
    for n, seed in ((4, 0), (10, 1), (40, 2), (100, 3)):
        e = I.random_planar_cubic_graph(n, seed)
        assert e == I.random_planar_cubic_graph(n, seed)
        g = nx.Graph(e)
        assert len(e) == 3 * n // 2 and g.number_of_edges() == len(e) and all(u != v for u, v in e)
        assert all(d == 3 for _, d in g.degree()) and nx.is_connected(g) and nx.check_planarity(g)[0]
    n = 160
    planar = [tnc.plan_formula(I.vertex_cover_formula(n, I.random_planar_cubic_graph(n, s)), heuristic="best",
                               rank_cap=64).stats.max_rank for s in range(3)]
    free = [tnc.plan_formula(I.cubic_vertex_cover(n, s), heuristic="best", rank_cap=64).stats.max_rank
            for s in range(3)]
    assert max(planar) + 8 <= min(free)
