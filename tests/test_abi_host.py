"""Host-side checks of libtnc (no GPU): exports, networks, planners, lowering."""
import ctypes
import math
import os
import re
import subprocess

import pytest

from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


def _declared():
    src = open(os.path.join(ROOT, "include", "tnc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*[\w\s\*]+?\b(tnc_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert len(names) >= 19
    out = subprocess.run(["nm", "-D", "--defined-only", tnc.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (tnc_\w+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(tnc.LIB_PATH)
    for n in names:
        assert hasattr(lib, n)
    assert sorted(tnc.EXPORTS) == names


def test_version_and_primes():
    assert "sm_103a" in tnc.version()
    p = tnc.default_primes(8)
    assert p[0] == 1073741789 and p == sorted(p, reverse=True) and len(set(p)) == 8  # largest below 2^30

    def isprime(n):
        if n < 2:
            return False
        i = 2
        while i * i <= n:
            if n % i == 0:
                return False
            i += 1
        return True
    # every odd number between 2^30 and p[0], and between consecutive primes, is composite
    for x in range(p[0] + 2, 2 ** 30, 2):
        assert not isprime(x)
    for a, b in zip(p, p[1:]):
        assert isprime(a) and isprime(b)
        for x in range(b + 2, a, 2):
            assert not isprime(x)


def test_p8_primes_and_options():
    """TNC_PATH_TC_P8: its default primes are the odd primes <= 251, largest
    first (checked by trial division); bad options are refused on the host."""
    odd_primes = [n for n in range(251, 2, -2) if all(n % d for d in range(3, int(n ** 0.5) + 1, 2))]
    assert len(odd_primes) == 53
    assert tnc.default_primes(53, "tc_p8") == odd_primes
    assert tnc.default_primes(5, "tc_p8") == [251, 241, 239, 233, 229]
    with pytest.raises(tnc.TncError):
        tnc.default_primes(54, "tc_p8")
    p = tnc.plan_formula(I.cubic_vertex_cover(30, 0))
    assert tnc.workspace_bytes(p, 20, "tc_p8") > 0
    assert tnc.workspace_bytes(p, 4, "int64") == tnc.lib().tnc_workspace_bytes(p.h, 4)
    for bad in ([257], [1], [4], [1073741789]):
        with pytest.raises(tnc.TncError):
            tnc.workspace_bytes(p, 1, "tc_p8", primes=bad)
    with pytest.raises(tnc.TncError):
        tnc.workspace_bytes(p, 54, "tc_p8")
    with pytest.raises(tnc.TncError):
        tnc.Batch([p], n_residues=4, path="tc_p8")


def test_p8_direct_plane_layout():
    """TNC_PATH_TC_P8 lays the arena out again: a dense step whose output
    feeds a dense step directly (as its fp16 operand planes) takes twice its
    entries, and the path's workspace covers that arena (4 residue bytes per
    entry in a pass of 4).  The lowering's own validation (every range inside
    the arena, no overlap within a level) runs at plan time."""
    p = tnc.plan_formula(I.cubic_vertex_cover(110, 6), heuristic="greedy", rank_cap=26)
    st = p.stats
    assert 1 <= st.n_direct_p8 < st.n_dense_steps_p8
    assert st.batch_arena_entries < st.p8_arena_entries <= 2 * st.batch_arena_entries
    assert tnc.workspace_bytes(p, 12, "tc_p8") >= 4 * st.p8_arena_entries
    q = tnc.plan_formula(I.cubic_vertex_cover(30, 0))  # no dense step: the same layout, 16-entry aligned
    assert q.stats.n_direct_p8 == 0
    assert q.stats.batch_arena_entries <= q.stats.p8_arena_entries <= 1.25 * q.stats.batch_arena_entries


def test_network_info_and_components():
    f = I.cubic_vertex_cover(20, 0)
    n, bonds, comps = tnc.build_network(f).info()
    assert (n, bonds, comps) == (20 + 30, 60, 1)
    g = I.Formula(7, [(0, 1), (2, 3)], [I.KIND_OR, I.KIND_OR])
    n, bonds, comps = tnc.build_network(g).info()
    assert (n, bonds) == (2 + 7, 4) and comps == 2 + 3  # two clause components + 3 lone vars


def test_invalid_formulas_are_rejected():
    with pytest.raises(tnc.TncError) as e:
        tnc.build_network(type("F", (), dict(n_vars=2, clauses=[(0, 5)], kinds=[1], tables=[None],
                                             open_vars=[]))())
    assert e.value.code == -1
    with pytest.raises(tnc.TncError):
        tnc.build_network(type("F", (), dict(n_vars=2, clauses=[(0, 1)], kinds=[9], tables=[None],
                                             open_vars=[]))())
    with pytest.raises(tnc.TncError):
        tnc.build_network(type("F", (), dict(n_vars=2, clauses=[(0, 1)], kinds=[1], tables=[None],
                                             open_vars=[0, 0]))())


@pytest.mark.parametrize("h", ["greedy", "bisect", "gn", "best", "coarsen"])
def test_planners_build_full_trees(h):
    f = I.cubic_vertex_cover(60, 3)
    p = tnc.plan(tnc.build_network(f), heuristic=h)
    steps = p.steps()
    L = f.n_vars + f.n_cons
    assert len(steps) == L - 1 == p.stats.n_steps
    used = set()
    for i, (a, b) in enumerate(steps):
        assert a < L + i and b < L + i and a != b
        assert a not in used and b not in used
        used |= {a, b}
    assert len(used) == 2 * (L - 1)
    assert 3 <= p.stats.max_rank <= 16


def test_explicit_order_is_kept():
    f = I.worked_example()
    order = [(0, 2), (1, 3), (6, 7), (4, 8), (5, 9)]  # ids as the oracle numbers them
    p = tnc.plan(tnc.build_network(f), order=order, n_open=2)
    assert p.steps() == order
    with pytest.raises(tnc.TncError):
        tnc.plan(tnc.build_network(f), order=[(0, 0)], n_open=2)


def test_rank_cap_reports_too_large():
    f = I.cubic_vertex_cover(60, 0)
    with pytest.raises(tnc.TncError) as e:
        tnc.plan(tnc.build_network(f), heuristic="greedy", rank_cap=6)
    assert e.value.code == -2


def test_lazy_cost_matches_definition():
    """Plan stats are the exact sum over steps of 2^(a+b-k) (Corollary 2 cost),
    recomputed here from the exported tree and the bond structure."""
    f = I.one_in_three(30, 18, 2)
    p = tnc.plan(tnc.build_network(f), heuristic="bisect")
    bonds = {}
    b = 0
    for c, vs in enumerate(f.clauses):
        for v in vs:
            bonds.setdefault(c, set()).add(b)
            bonds.setdefault(f.n_cons + v, set()).add(b)
            b += 1
    for t in range(f.n_cons + f.n_vars):
        bonds.setdefault(t, set())
    macs, mx = 0, max(len(s) for s in bonds.values())
    nxt = f.n_cons + f.n_vars
    for a, c in p.steps():
        A, B = bonds.pop(a), bonds.pop(c)
        k = len(A & B)
        macs += 2 ** (len(A) + len(B) - k)
        bonds[nxt] = A ^ B
        mx = max(mx, len(A ^ B))
        nxt += 1
    assert math.isclose(p.stats.total_macs, macs) and p.stats.max_rank == mx


def test_bound_certifies_small_counts():
    import oracle
    for s in range(5):
        f = I.one_in_three(40, 25, s)
        p = tnc.plan(tnc.build_network(f), heuristic="greedy")
        z = oracle.count(f)[0]
        assert z <= 2 ** p.stats.log2_bound + 1e-6


DEGENERATE = [
    I.Formula(1, [], []),
    I.Formula(0, [], []),
    I.Formula(3, [(0, 1, 2), ()], [I.KIND_1IN3, I.KIND_OR]),
    I.Formula(5, [(0, 1, 2)], [I.KIND_1IN3]),
    I.Formula(4, [(0, 1)], [I.KIND_OR], open_vars=[3, 0]),
    I.Formula(6, [(0, 1), (2, 3), (4, 5)], [I.KIND_NAND] * 3),
    I.Formula(2, [()], [I.KIND_TABLE], tables=[[7]]),
    I.Formula(3, [(0,), (1,), (2,)], [I.KIND_OR] * 3, open_vars=[0, 1, 2]),
]


@pytest.mark.parametrize("h", ["greedy", "bisect", "gn", "best", "coarsen"])
def test_degenerate_formulas_plan(h):
    for f in DEGENERATE:
        p = tnc.plan_formula(f, heuristic=h)
        assert p.stats.n_steps == max(f.n_vars + f.n_cons - 1, 0)
    tnc.plan_many(DEGENERATE, heuristic=h)


def test_coarsen_plan_is_never_costlier_than_the_whole_network_heuristics():
    """TNC_PLAN_COARSEN keeps the fewest MACs within the rank cap among
    candidates that include tensor-greedy, tensor-METIS (same tries and seed)
    and tensor-GN planned on the whole network (Sec. 3.1.1), so within the
    cap it never needs more MACs than any of the three."""
    forms = [I.cubic_vertex_cover(60, s) for s in range(6)] + \
        [I.one_in_three(100, 62, s) for s in range(4)]
    gains = []
    for f in forms:
        net = tnc.build_network(f)
        c = tnc.plan(net, heuristic="coarsen", rank_cap=32)
        assert c.stats.max_rank <= 32
        others = [tnc.plan(net, heuristic=h, rank_cap=64) for h in ("greedy", "bisect", "gn")]
        fit = [o.stats.total_macs for o in others if o.stats.max_rank <= 32]
        assert fit and c.stats.total_macs <= min(fit)
        gains.append(min(fit) / c.stats.total_macs)
    # the coarsened candidates do win on these workloads, not only tie
    assert sum(g > 1.0 for g in gains) >= len(forms) // 2


def test_coarsen_order_gives_the_oracle_count():
    """The oracle contracting along the coarsen plan's own order (an explicit
    pairwise order) gets the count it gets along its default order: the plan
    is a full, valid contraction tree."""
    import oracle
    for f in (I.cubic_vertex_cover(40, 1), I.one_in_three(40, 26, 2), I.worked_example()):
        p = tnc.plan_formula(f, heuristic="coarsen")
        assert oracle.count(f, order=p.steps(), max_rank=26) == oracle.count(f, max_rank=26)
