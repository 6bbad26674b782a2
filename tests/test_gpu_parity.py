"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact: every residue must equal the oracle's exact count mod that prime,
and every CRT value must equal the exact count whenever it is certified below
the product of the primes.
"""
import random

import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc
from _util import random_formula, random_order

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


def _check(res: tnc.Count, exact, R):
    assert len(res.counts) == len(exact)
    for e, z in enumerate(exact):
        assert [int(x) for x in res.residues[e]] == [z % p for p in res.primes], (e, z)
    prod = 1
    for p in res.primes:
        prod *= p
    if not res.flags & tnc.TNC_MAYBE_WRAPPED:
        assert res.counts == list(exact)
    else:
        assert res.counts == [z % prod for z in exact]


def test_worked_example_open_bonds():
    f = I.worked_example()
    for h in ("greedy", "bisect", "gn"):
        r = tnc.contract(tnc.plan_formula(f, heuristic=h), n_residues=2)
        assert r.counts == [3, 3, 3, 4]


@pytest.mark.parametrize("seed", range(8))
def test_one_in_three_n20_bruteforce(seed):
    f = I.one_in_three(20, 12, seed)
    exact = oracle.bruteforce(f)
    for h in ("greedy", "bisect", "gn"):
        for R in (1, 2):
            _check(tnc.contract(tnc.plan_formula(f, heuristic=h), n_residues=R), exact, R)


@pytest.mark.parametrize("seed", range(6))
def test_cubic_vc_n60_four_residues(seed):
    f = I.cubic_vertex_cover(60, seed)
    exact = oracle.count(f)
    for h in ("bisect", "gn", "coarsen"):
        r = tnc.contract(tnc.plan_formula(f, heuristic=h), n_residues=4)
        _check(r, exact, 4)
        assert r.flags == 0 and r.counts == exact


def test_count_above_2_64_lucas():
    f = I.vertex_cover_formula(130, I.cycle_graph(130))
    exact = oracle.count(f)
    assert exact[0] > 2 ** 64
    for R in (3, 4, 5, 8):
        _check(tnc.contract(tnc.plan_formula(f, heuristic="bisect"), n_residues=R), exact, R)


def test_wrapped_flag_with_one_prime():
    f = I.cubic_vertex_cover(60, 1)
    r = tnc.contract(tnc.plan_formula(f, heuristic="gn"), n_residues=1)
    exact = oracle.count(f)
    assert r.flags & tnc.TNC_MAYBE_WRAPPED
    _check(r, exact, 1)


@pytest.mark.parametrize("seed", range(12))
def test_random_formulas_all_kinds(seed):
    rng = random.Random(seed)
    n = rng.randint(1, 16)
    f = random_formula(rng, n, rng.randint(0, 14), rng.randint(0, min(4, n)),
                       weights=(0, 1, 2, 7, 2 ** 32 - 1), allow_empty=True)
    exact = oracle.bruteforce(f)
    for h in ("greedy", "bisect", "gn"):
        _check(tnc.contract(tnc.plan_formula(f, heuristic=h), n_residues=4), exact, 4)


def test_degenerate_formulas():
    cases = [
        I.Formula(1, [], []),                              # one free variable: 2
        I.Formula(0, [], []),                              # empty: 1
        I.Formula(3, [(0, 1, 2), ()], [I.KIND_1IN3, I.KIND_OR]),  # empty OR clause: 0
        I.Formula(5, [(0, 1, 2)], [I.KIND_1IN3]),          # unused variables
        I.Formula(4, [(0, 1)], [I.KIND_OR], open_vars=[3, 0]),  # open var in no clause
        I.Formula(6, [(0, 1), (2, 3), (4, 5)], [I.KIND_NAND] * 3),  # components
    ]
    for f in cases:
        exact = oracle.bruteforce(f)
        r = tnc.contract(tnc.plan_formula(f, heuristic="greedy"), n_residues=2)
        assert r.counts == exact, (f.clauses, r.counts, exact)


def test_random_orders_agree():
    """Order independence on the device: random explicit orders, one count."""
    rng = random.Random(5)
    f = I.cubic_vertex_cover(24, 2)
    exact = oracle.count(f)
    for _ in range(10):
        p = tnc.plan(tnc.build_network(f), order=random_order(rng, f), rank_cap=26)
        assert tnc.contract(p, n_residues=2).counts == exact


@pytest.mark.parametrize("R", [1, 2, 4, 6])
def test_batch_matches_oracle_and_replays(R):
    import torch
    forms = [I.cubic_vertex_cover(60, s) for s in range(24)] + [I.one_in_three(40, 26, s) for s in range(24)]
    forms += [I.worked_example(), I.Formula(1, [], []), random_formula(random.Random(3), 10, 9, 2)]
    plans = [tnc.plan_formula(f, heuristic="gn") for f in forms]
    exact = [oracle.count(f) for f in forms]
    b = tnc.Batch(plans, n_residues=R)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    b.upload(ws, stream)
    for rep in range(3):  # first launch captures the graph, the others replay it
        b.launch(ws, stream)
        out = b.download(ws, stream)
        for r, z in zip(out, exact):
            _check(r, z, R)
    res, limbs, flags = b.download_flat(ws, stream)  # bulk form, formula after formula
    e = 0
    for f, r, z in zip(forms, out, exact):
        n = 1 << len(f.open_vars)
        assert res[e:e + n].tolist() == r.residues.tolist()
        assert tnc.Batch.counts_from_limbs(limbs[e:e + n]) == r.counts
        e += n
    assert e == res.shape[0] and flags.tolist() == [r.flags for r in out]
    ws2 = torch.full_like(ws, 0x5A)  # stale garbage everywhere: results must not depend on it
    b.upload(ws2, stream)
    b.launch(ws2, stream)
    for r, z in zip(b.download(ws2, stream), exact):
        _check(r, z, R)
    out2 = tnc.contract_batch(plans, n_residues=R)
    for r, z in zip(out2, exact):
        _check(r, z, R)


def test_prism_180_vertices_closed_form():
    """A cubic graph on 180 vertices (the large VC size) with a closed-form
    count: prism with 90 rungs, #IS = trace(T^90); needs 8 residues."""
    n = 90
    T = [[1, 1, 1], [1, 0, 1], [1, 1, 0]]
    R_ = [[int(i == j) for j in range(3)] for i in range(3)]
    for _ in range(n):
        R_ = [[sum(R_[i][k] * T[k][j] for k in range(3)) for j in range(3)] for i in range(3)]
    want = sum(R_[i][i] for i in range(3))
    f = I.independent_set_formula(2 * n, I.prism_graph(n))
    r = tnc.contract(tnc.plan_formula(f, heuristic="bisect"), n_residues=8)
    assert r.counts == [want] and r.flags == 0


def test_batches_with_different_descriptor_sizes_coexist():
    """The batch kernel's shared-memory limit is per kernel, not per batch: a
    batch with large descriptors still launches after a batch with small
    descriptors was created (and configured) after it."""
    import torch
    big_f = [I.cubic_vertex_cover(70, s) for s in range(6)]
    small_f = [I.one_in_three(12, 6, s) for s in range(6)]
    big = tnc.Batch([tnc.plan_formula(f, heuristic="best") for f in big_f], n_residues=4)
    small = tnc.Batch([tnc.plan_formula(f, heuristic="best") for f in small_f], n_residues=4)
    stream = torch.cuda.Stream()
    for b, fs in ((big, big_f), (small, small_f), (big, big_f)):
        ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device="cuda")
        b.upload(ws, stream)
        b.launch(ws, stream)
        for r, f in zip(b.download(ws, stream), fs):
            _check(r, oracle.count(f), 4)


# caller-supplied primes: near 2^31 (a reduction every 4 products), below
# 2^30 - 2^10 (the Barrett reduction for every group), and groups mixing
# them with primes just below 2^30 (whose groups otherwise take the two-fold
# reduction)
USER_PRIMES = {
    "near_2_31": [2147483647, 2147483629, 2147483587, 2147483579],
    "mid": [1073740793, 1073740783, 1073740781, 537919441],
    "mixed_group": [1073741789, 2147483647, 1073741783, 1073740793, 2147483629],
    "groups_of_both": [1073741789, 1073741783, 1073741741, 1073741723, 2147483647, 1073740793],
}


@pytest.mark.parametrize("which", sorted(USER_PRIMES))
def test_user_primes_int64_and_batch(which):
    import torch
    primes = USER_PRIMES[which]
    forms = [I.cubic_vertex_cover(70, s) for s in range(3)] + [I.one_in_three(30, 19, 7), I.worked_example()]
    plans = [tnc.plan_formula(f, heuristic="best") for f in forms]
    exact = [oracle.count(f) for f in forms]
    for p, z in zip(plans, exact):
        r = tnc.contract(p, n_residues=len(primes), primes=primes)
        assert r.primes == primes
        _check(r, z, len(primes))
    b = tnc.Batch(plans, n_residues=len(primes), primes=primes)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    b.upload(ws, stream)
    b.launch(ws, stream)
    for r, z in zip(b.download(ws, stream), exact):
        _check(r, z, len(primes))


def test_autotune_choice_is_persisted_and_reused(tmp_path):
    """The autotuned launch shape is written to a JSON file keyed by device
    and batch sizes; a second batch of the same sizes reads it back (no
    timing) and counts the same."""
    import json
    import torch
    forms = [I.cubic_vertex_cover(40, s) for s in range(64)]
    plans = tnc.plan_many(forms, heuristic="gn")
    cache = str(tmp_path / "tune.json")
    st = torch.cuda.Stream()
    b1 = tnc.Batch(plans, n_residues=2)
    ws = torch.empty(b1.workspace_bytes(), dtype=torch.uint8, device="cuda")
    b1.upload(ws, st)
    shape1 = b1.autotune_cached(ws, st, cache=cache)
    assert tuple(shape1) == b1.get_launch()
    table = json.load(open(cache))
    assert list(table.values()) == [list(shape1)]
    b2 = tnc.Batch(plans, n_residues=2)
    b2.upload(ws, st)
    assert tuple(b2.autotune_cached(ws, st, cache=cache)) == tuple(shape1) == b2.get_launch()
    b2.launch(ws, st)
    assert [o.counts for o in b2.download(ws, st)] == [oracle.count(f) for f in forms]
