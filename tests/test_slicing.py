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
    plans, vs = S.sliced_plans(f, 3)
    assert len(plans) == 8 and len(set(vs)) == 3
    assert max(p.stats.max_rank for p in plans) <= full.stats.max_rank - 2
    assert max(p.stats.arena_entries for p in plans) * 4 <= full.stats.arena_entries


@pytest.mark.parametrize("seed", [3, 15])
def test_slicing_cost_never_grows_with_s(seed):
    """Each added slice variable is chosen by the exact plan cost of its
    slices (the current plan restricted to a slice is always a candidate):
    the max rank and the total MACs of all slices do not grow with s."""
    f = I.cubic_vertex_cover(180, seed)
    prev = None
    for s in range(5):
        plans, vs = S.sliced_plans(f, s)
        assert len(plans) == 2 ** s and len(set(vs)) == s
        cost = (max(p.stats.max_rank for p in plans), sum(p.stats.total_macs for p in plans))
        if prev is not None:
            assert cost[0] <= prev[0] and cost[1] <= prev[1] * (1 + 1e-12), (s, cost, prev)
        prev = cost


def test_library_slices_match_the_definition():
    """tnc_slice_network's restricted clause tables, read back, are the clause
    tensors with the fixed bonds set (checked entry by entry against the
    definitions of Eq. 1in3, Eq. or and NAND)."""
    rng = random.Random(5)
    f = random_formula(rng, 10, 8)
    g = S.slice_formula(f, {2: 1, 5: 0})
    keep = [v for v in range(f.n_vars) if v not in (2, 5)]
    assert g.n_vars == 8 and len(g.clauses) == len(f.clauses)
    fixed = {2: 1, 5: 0}
    for c, k, t, gc, gk, gt in zip(f.clauses, f.kinds, f.tables, g.clauses, g.kinds, g.tables):
        free = [v for v in c if v not in fixed]
        assert list(gc) == [keep.index(v) for v in free]
        if len(free) == len(c):
            assert gk == k
            continue
        assert gk == I.KIND_TABLE
        for j in range(1 << len(free)):
            val = dict(fixed)
            val.update({v: (j >> i) & 1 for i, v in enumerate(free)})
            idx = sum(val[v] << i for i, v in enumerate(c))
            ones = bin(idx).count("1")
            want = {I.KIND_1IN3: int(ones == 1), I.KIND_OR: int(idx != 0),
                    I.KIND_NAND: int(idx != (1 << len(c)) - 1)}.get(k, None)
            assert gt[j] == (t[idx] if k == I.KIND_TABLE else want)


def test_library_rejects_slicing_an_open_variable():
    f = I.one_in_three(16, 10, 3)
    f.open_vars = [4]
    arr = tnc.np.array([4], dtype=tnc.np.int32)
    h = tnc.ctypes.c_void_p()
    net = tnc.build_network(f)
    rc = tnc.lib().tnc_slice_network(net.h, 1, tnc._p(arr, tnc.ctypes.c_int32), 0, tnc.ctypes.byref(h))
    assert rc == -1


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
