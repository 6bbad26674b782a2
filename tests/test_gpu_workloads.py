"""GPU parity on the workloads beyond the benchmark configurations: the
paper's own 1-in-3 distribution (variables are the edges of a random cubic
graph, so the count is its number of perfect matchings) and general CNF with
negated literals (TABLE clause tensors).  Every arithmetic path against the
CPU oracle, bit for bit."""
import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


def _perfect_matchings(n, edges):
    """Perfect matchings of a small graph by recursion on the lowest vertex."""
    adj = {v: [] for v in range(n)}
    for i, (u, v) in enumerate(edges):
        adj[u].append((v, i))
        adj[v].append((u, i))

    def rec(free):
        if not free:
            return 1
        v = min(free)
        return sum(rec(free - {v, u}) for u, _ in adj[v] if u in free)
    return rec(frozenset(range(n)))


@pytest.mark.parametrize("seed", range(4))
def test_cubic_one_in_three_is_perfect_matchings(seed):
    f = I.cubic_one_in_three(16, seed)
    edges = I.random_cubic_graph(16, seed)
    pm = _perfect_matchings(16, edges)
    for path in ("int64", "tc", "tc_p8"):
        p = tnc.plan_formula(f, heuristic="best")
        R = 8 if path == "tc_p8" else 2
        assert tnc.contract(p, n_residues=R, path=path).counts == [pm]


@pytest.mark.parametrize("nv", [40, 60, 80])
def test_cubic_one_in_three_batch_matches_oracle(nv):
    forms = [I.cubic_one_in_three(nv, s) for s in range(24)]
    plans = tnc.plan_many(forms, heuristic="best")
    got = tnc.contract_batch(plans, n_residues=2)
    for f, r in zip(forms, got):
        assert r.counts == oracle.count(f)


@pytest.mark.parametrize("n,m", [(40, 24), (60, 40), (80, 52)])
def test_cnf_with_negations_all_paths(n, m):
    for seed in range(3):
        f = I.random_k_cnf(n, m, 3, seed)
        exact = oracle.count(f, max_rank=28)
        p = tnc.plan_formula(f, heuristic="best", rank_cap=28)
        for path, R in (("int64", 3), ("tc", 3), ("tc_p8", 12)):
            r = tnc.contract(p, n_residues=R, path=path)
            assert r.counts == exact and r.flags == 0


def test_cnf_batch_matches_oracle():
    forms = [I.random_k_cnf(60, 40, 3, 100 + s) for s in range(32)]
    plans = tnc.plan_many(forms, heuristic="best")
    got = tnc.contract_batch(plans, n_residues=2)
    for f, r in zip(forms, got):
        assert r.counts == oracle.count(f)
