"""Pins of the CPU oracle against facts fixed outside it (paper, textbook, hand).

Each test pins both oracle routes (C brute force, C contraction) and, where
small, the pure-Python twin.  A dropped term, a wrong clause definition or a
transposed open index fails at least one of them.
"""
import json
import os
import random

import pytest

import oracle
from oracle.pyoracle import py_bruteforce, py_contract
from paper_1805_00475_gb300 import instances as I
from _util import random_order

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- the paper's example

def test_worked_example_matrix():
    """Sec. 2.1 worked contraction: ((3,3),(3,4)) over the open legs (i1, i6)."""
    g = _gold("worked_example.json")
    kinds = {"OR": I.KIND_OR}
    f = I.Formula(g["n_vars"], [tuple(c) for c in g["clauses"]], [kinds[k] for k in g["kinds"]],
                  open_vars=g["open_vars"])
    exp = g["expected_matrix_i1_i6"]
    flat = [exp[i1][i6] for i6 in (0, 1) for i1 in (0, 1)]  # index i1 + 2*i6
    assert oracle.count(f) == flat
    assert oracle.bruteforce(f) == flat
    assert py_contract(f) == flat
    assert py_bruteforce(f) == flat
    # the example is symmetric except at (1,1); swapping the open order must keep it
    f2 = I.Formula(4, f.clauses, f.kinds, open_vars=[3, 2])
    assert oracle.count(f2) == flat


def test_open_index_order_is_not_symmetric():
    """An asymmetric open tensor pins the open-bond bit order (index bit i =
    open variable i): with x0 forced to 1 by a unit OR clause, T[x0, x1] is
    nonzero only at x0=1."""
    f = I.Formula(2, [(0,), (0, 1)], [I.KIND_OR, I.KIND_OR], open_vars=[0, 1])
    # x0=1 satisfies both for any x1 -> entries (1,0),(1,1) are 1; x0=0 -> 0
    expect = [0, 1, 0, 1]  # index x0 + 2*x1
    assert oracle.count(f) == expect
    assert oracle.bruteforce(f) == expect
    assert py_contract(f) == expect


# ---------------------------------------------------------------- hand counts

def test_k4_vertex_cover_is_5():
    g = _gold("hand_counts.json")
    f = I.vertex_cover_formula(4, I.complete_graph(4))
    assert oracle.count(f) == [g["k4_vertex_covers"]["value"]]
    assert oracle.bruteforce(f) == [5]
    assert py_contract(f) == [5]


def test_perfect_matchings_k4_k33():
    """Monotone 1-in-3 with clauses on vertices, variables on edges counts
    perfect matchings (Sec. 3.2): K4 -> 3, K_{3,3} -> 6."""
    g = _gold("hand_counts.json")
    for edges, nv, key in ((I.complete_graph(4), 4, "k4_perfect_matchings"),
                           (I.complete_bipartite(3, 3), 6, "k33_perfect_matchings")):
        inc = [[] for _ in range(nv)]
        for i, (u, v) in enumerate(edges):
            inc[u].append(i)
            inc[v].append(i)
        f = I.Formula(len(edges), [tuple(c) for c in inc], [I.KIND_1IN3] * nv)
        want = g[key]["value"]
        assert oracle.count(f) == [want]
        assert oracle.bruteforce(f) == [want]


def test_prism3_independent_sets_is_13():
    f = I.independent_set_formula(6, I.prism_graph(3))
    assert oracle.count(f) == [13] and oracle.bruteforce(f) == [13]


# ---------------------------------------------------------------- closed forms

def _lucas(n):
    a, b = 2, 1
    for _ in range(n):
        a, b = b, a + b
    return a


def _trace_pow(T, n):
    dim = len(T)
    R = [[int(i == j) for j in range(dim)] for i in range(dim)]
    for _ in range(n):
        R = [[sum(R[i][k] * T[k][j] for k in range(dim)) for j in range(dim)] for i in range(dim)]
    return sum(R[i][i] for i in range(dim))


@pytest.mark.parametrize("n", [3, 4, 5, 10, 31, 64, 97, 130])
def test_cycle_vertex_covers_are_lucas(n):
    """#VC(C_n) = #IS(C_n) = L_n (transfer matrix [[1,1],[1,0]]); exceeds 2^64 at n >= 93."""
    vc = oracle.count(I.vertex_cover_formula(n, I.cycle_graph(n)))
    is_ = oracle.count(I.independent_set_formula(n, I.cycle_graph(n)))
    assert vc == [_lucas(n)] and is_ == [_lucas(n)]
    if n <= 16:
        assert oracle.bruteforce(I.vertex_cover_formula(n, I.cycle_graph(n))) == [_lucas(n)]


@pytest.mark.parametrize("n", [3, 4, 7, 20, 50])
def test_prism_independent_sets_transfer_matrix(n):
    T = [[1, 1, 1], [1, 0, 1], [1, 1, 0]]
    f = I.independent_set_formula(2 * n, I.prism_graph(n))
    assert oracle.count(f) == [_trace_pow(T, n)]


def test_disjoint_one_in_three_clauses():
    """m vertex-disjoint 1-in-3 clauses and `free` unused variables: 3^m * 2^free."""
    for m, free in ((1, 0), (4, 3), (9, 5), (30, 7)):
        n = 3 * m + free
        f = I.Formula(n, [(3 * i, 3 * i + 1, 3 * i + 2) for i in range(m)], [I.KIND_1IN3] * m)
        assert oracle.count(f) == [3 ** m * 2 ** free]
        if n <= 20:
            assert oracle.bruteforce(f) == [3 ** m * 2 ** free]


def test_empty_formula_counts_all_assignments():
    for n in (0, 1, 5):
        f = I.Formula(n, [], [])
        assert oracle.count(f) == [2 ** n]
        assert oracle.bruteforce(f) == [2 ** n]


# ---------------------------------------------------------------- equivalences

@pytest.mark.parametrize("seed", range(6))
def test_vc_equals_is_on_cubic_graphs(seed):
    """Complement bijection: #VC(G) = #IS(G) on the same graph."""
    n = 12 + 2 * seed
    e = I.random_cubic_graph(n, seed)
    assert oracle.count(I.vertex_cover_formula(n, e)) == oracle.count(I.independent_set_formula(n, e))


def _ryser_permanent(M):
    n = len(M)
    total = 0
    for S in range(1, 1 << n):
        prod = 1
        for i in range(n):
            prod *= sum(M[i][j] for j in range(n) if (S >> j) & 1)
        total += (-1) ** bin(S).count("1") * prod
    return (-1) ** n * total


def test_bipartite_cubic_one_in_three_is_permanent():
    """On bipartite cubic graphs, 1-in-3 with variables on edges = perfect
    matchings = permanent of the biadjacency matrix (Ryser's formula)."""
    rng = random.Random(7)
    for side in (4, 5, 6, 7):
        # union of 3 random perfect matchings without repeats -> 3-regular bipartite
        while True:
            perms = [list(range(side)) for _ in range(3)]
            for p in perms:
                rng.shuffle(p)
            edges = {(i, side + p[i]) for p in perms for i in range(side)}
            if len(edges) == 3 * side:
                break
        edges = sorted(edges)
        M = [[0] * side for _ in range(side)]
        for u, v in edges:
            M[u][v - side] = 1
        inc = [[] for _ in range(2 * side)]
        for i, (u, v) in enumerate(edges):
            inc[u].append(i)
            inc[v].append(i)
        f = I.Formula(len(edges), [tuple(c) for c in inc], [I.KIND_1IN3] * (2 * side))
        assert oracle.count(f) == [_ryser_permanent(M)]


def test_one_in_three_matches_its_cnf():
    """Eq. 1in3 equals the 5-clause CNF of Sec. 3.2 (as a TABLE of ORs of
    literals): brute force over both encodings agrees."""
    f = I.one_in_three(9, 5, 3)
    cnf_table = []
    for idx in range(8):
        x = [(idx >> j) & 1 for j in range(3)]
        ok = ((x[0] or x[1] or x[2]) and (x[0] or not x[1] or not x[2]) and
              (not x[0] or not x[1] or x[2]) and (not x[0] or x[1] or not x[2]) and
              (not x[0] or not x[1] or not x[2]))
        cnf_table.append(int(bool(ok)))
    g = I.Formula(f.n_vars, f.clauses, [I.KIND_TABLE] * f.n_cons, tables=[cnf_table] * f.n_cons)
    assert oracle.bruteforce(f) == oracle.bruteforce(g) == oracle.count(g)


# ---------------------------------------------------------------- random cross-checks

def _random_formula(rng, n, m, n_open=0):
    clauses, kinds, tables = [], [], []
    for _ in range(m):
        d = rng.randint(1, 4)
        vs = tuple(rng.sample(range(n), min(d, n)))
        k = rng.choice([I.KIND_1IN3, I.KIND_OR, I.KIND_NAND, I.KIND_TABLE])
        clauses.append(vs)
        kinds.append(k)
        tables.append([rng.randint(0, 5) for _ in range(1 << len(vs))] if k == I.KIND_TABLE else None)
    opens = rng.sample(range(n), n_open)
    return I.Formula(n, clauses, kinds, tables, open_vars=opens)


@pytest.mark.parametrize("seed", range(20))
def test_contract_equals_bruteforce_random(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 14)
    f = _random_formula(rng, n, rng.randint(0, 12), rng.randint(0, min(3, n)))
    bf = oracle.bruteforce(f)
    assert oracle.count(f) == bf
    assert py_bruteforce(f) == bf
    if n <= 8:
        assert py_contract(f) == bf


@pytest.mark.parametrize("seed", range(10))
def test_order_independence(seed):
    """The full trace does not depend on the contraction order (Sec. 2.1)."""
    rng = random.Random(100 + seed)
    f = I.one_in_three(24, 16, seed) if seed % 2 else I.cubic_vertex_cover(20, seed)
    ref = oracle.count(f)
    for _ in range(3):
        assert oracle.count(f, order=random_order(rng, f), max_rank=26) == ref
    if f.n_vars <= 24:
        assert oracle.bruteforce(f) == ref


def test_config_one_in_three_n20_bruteforce():
    """Monotone 1-in-3, n=20, m=12 (the small brute-force-checkable case)."""
    for seed in range(10):
        f = I.one_in_three(20, 12, seed)
        assert oracle.count(f) == oracle.bruteforce(f)


def test_contract_rejects_bad_order():
    f = I.one_in_three(6, 2, 0)
    with pytest.raises(RuntimeError):
        oracle.count(f, order=[(0, 0)])
    with pytest.raises(RuntimeError):
        oracle.count(f, order=[(0, 99)])


def _cnf_bruteforce(n, lit_clauses):
    """Satisfying assignments of a CNF evaluated literal by literal (no clause
    tensors involved)."""
    total = 0
    for x in range(1 << n):
        if all(any(((x >> (abs(l) - 1)) & 1) == (1 if l > 0 else 0) for l in c) for c in lit_clauses):
            total += 1
    return total


def _cnf_literals(n, m, k, seed):
    rng = random.Random(seed)
    return [[rng.choice([1, -1]) * (v + 1) for v in rng.sample(range(n), k)] for _ in range(m)]


@pytest.mark.parametrize("seed", range(6))
def test_cnf_with_negations_matches_literal_bruteforce(seed):
    """General CNF (negated literals as reversed bond indices, Sec. 2.1): the
    oracle's contraction equals the count of assignments satisfying every
    clause, evaluated directly on the literals."""
    n, lits = 13, _cnf_literals(13, 20, 3, seed)
    f = I.cnf_formula(n, lits)
    assert oracle.count(f) == [_cnf_bruteforce(n, lits)]


def test_cnf_count_invariant_under_flipping_a_variable():
    """Negating every literal of one variable permutes the assignments: the
    count is unchanged (and a clause with x and not x changes nothing)."""
    lits = _cnf_literals(12, 18, 3, 99)
    base = oracle.count(I.cnf_formula(12, lits))
    for v in (1, 5, 12):
        flipped = [[-l if abs(l) == v else l for l in c] for c in lits]
        assert oracle.count(I.cnf_formula(12, flipped)) == base
    assert oracle.count(I.cnf_formula(12, lits + [[3, -3, 7]])) == base


def test_positive_cnf_equals_or_clauses():
    """A CNF without negations is the OR-clause formula of the same scopes."""
    lits = [[abs(l) for l in c] for c in _cnf_literals(14, 12, 3, 7)]
    f_or = I.Formula(14, [tuple(abs(l) - 1 for l in c) for c in lits], [I.KIND_OR] * len(lits))
    assert oracle.count(I.cnf_formula(14, lits)) == oracle.count(f_or)
