"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The oracle cannot count every formula of a full benchmark batch in test time,
so a seeded sample of formulas is counted by the oracle and compared residue
by residue (and by CRT value where the count is certified) with what the
single persistent launch produced for them; every formula of the batch is
checked for internal consistency (its CRT value reduces to its residues).
"""
import random

import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


def _run_batch(plans, R):
    import torch
    b = tnc.Batch(plans, n_residues=R)
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.Stream()
    b.upload(ws, stream)
    b.autotune(ws, stream)  # the shape the benchmark launches
    b.launch(ws, stream)
    return b.download(ws, stream)


def _check_sample(out, forms, idx, order_of=None):
    for i in idx:
        f, r = forms[i], out[i]
        z = oracle.count(f, order_of(i) if order_of else None)
        assert [int(x) for x in r.residues[0]] == [z[0] % p for p in r.primes], i
        prod = 1
        for p in r.primes:
            prod *= p
        assert r.counts == ([z[0]] if not r.flags & tnc.TNC_MAYBE_WRAPPED else [z[0] % prod]), i


def _check_consistent(out):
    for r in out:
        for e, c in enumerate(r.counts):
            assert [c % p for p in r.primes] == [int(x) for x in r.residues[e]]


@pytest.mark.parametrize("planner", ["coarsen", "best"])
def test_c2_full_batch_sampled_against_oracle(planner):
    """#Cubic-Vertex-Cover on 60 vertices, seeds 0..8191, 4 residues below
    2^30: the default benchmark's 8192 formulas in one autotuned persistent
    launch, planned as the benchmark plans them (two-level plans) and by the
    best of the paper's heuristics; 64 sampled formulas plus the first and
    the last against the oracle."""
    forms = [I.cubic_vertex_cover(60, s) for s in range(8192)]
    plans = tnc.plan_many(forms, heuristic=planner)
    out = _run_batch(plans, 4)
    assert len(out) == 8192
    assert all(r.flags == 0 for r in out)  # 4 residues certify every count (bound <= 2^60)
    _check_consistent(out)
    idx = sorted(set(random.Random(8192).sample(range(8192), 64) + [0, 8191]))
    _check_sample(out, forms, idx)


def test_c3_batched_part_sampled_against_oracle():
    """The 4096 uneven monotone 1-in-3 formulas (n ~ U{50..150}, m/n ~
    U[0.5, 0.8)); those whose best plan has at most 2^24 MACs and rank <= 16
    go through one persistent launch with 2 residues, as in the benchmark.
    48 sampled formulas plus the first and the last batched one against the
    oracle, which contracts along the same tree (its count does not depend on
    the order: pinned on the CPU)."""
    forms = I.batch_one_in_three(4096, 2026)
    plans = tnc.plan_many(forms, heuristic="best", rank_cap=64)
    light = [i for i, p in enumerate(plans) if p.stats.total_macs <= 2.0 ** 24 and p.stats.max_rank <= 16]
    assert len(light) > 2000
    out = _run_batch([plans[i] for i in light], 2)
    _check_consistent(out)
    sub = [forms[i] for i in light]
    idx = sorted(set(random.Random(4096).sample(range(len(light)), 48) + [0, len(light) - 1]))
    _check_sample(out, sub, idx, order_of=lambda j: plans[light[j]].steps())


def _c3_heavy():
    """The benchmark's heavy 1-in-3 formulas: plans above 2^24 MACs or rank
    16, re-planned by the portfolio of the paper's heuristics."""
    forms = I.batch_one_in_three(4096, 2026)
    plans = tnc.plan_many(forms, heuristic="best", rank_cap=64)
    heavy = [i for i, p in enumerate(plans) if not (p.stats.total_macs <= 2.0 ** 24 and p.stats.max_rank <= 16)]
    hp = tnc.plan_many([forms[i] for i in heavy], heuristic="portfolio", rank_cap=64)
    return forms, heavy, hp


def test_c3_heavy_part_sampled_against_oracle():
    """All heavy formulas of rank <= 26 in one tnc_contract_many call (8 primes
    <= 251, as the benchmark): every CRT value consistent with its residues;
    24 sampled formulas (those of at most 2^30 MACs) against the oracle."""
    import torch
    forms, heavy, hp = _c3_heavy()
    sel = [j for j, p in enumerate(hp) if p.stats.max_rank <= 26]
    assert len(sel) > 1500
    plans = [hp[j] for j in sel]
    ws = torch.empty(16 << 30, dtype=torch.uint8, device="cuda")
    out = tnc.contract_many(plans, n_residues=8, path="tc_p8", workspace=ws)
    _check_consistent(out)
    small = [k for k, p in enumerate(plans) if p.stats.total_macs <= 2.0 ** 30]
    idx = sorted(random.Random(26).sample(small, 24))
    sub = [forms[heavy[sel[k]]] for k in range(len(sel))]
    _check_sample(out, sub, idx, order_of=lambda k: plans[k].steps())


def test_c3_sliced_part_equals_unsliced():
    """Formulas whose portfolio plan is above rank 26 are sliced to rank <= 26
    (tnc_plan_sliced); on two of them the sliced count equals the unsliced
    count of the 8-bit-prime path, and a disjoint set of primes rebuilds the
    same integer."""
    from paper_1805_00475_gb300 import slicing as S
    forms, heavy, hp = _c3_heavy()
    big = sorted((p.stats.total_macs, heavy[j]) for j, p in enumerate(hp) if 26 < p.stats.max_rank <= 29)[:2]
    assert len(big) == 2
    primes_a = tnc.default_primes(16, "tc_p8")
    primes_b = tnc.default_primes(32, "tc_p8")[16:]
    for _, i in big:
        s = 1
        while True:
            sp, vs = S.sliced_plans(forms[i], s, heuristic="best")
            if max(q.stats.max_rank for q in sp) <= 26:
                break
            s += 1
        whole = tnc.plan_formula(forms[i], heuristic="portfolio", rank_cap=30)
        a = tnc.contract(whole, n_residues=16, primes=primes_a, path="tc_p8")
        b = tnc.contract_sliced(sp, n_residues=16, primes=primes_a, path="tc_p8")
        c = tnc.contract_sliced(sp, n_residues=16, primes=primes_b, path="tc_p8")
        assert a.residues.tolist() == b.residues.tolist()
        assert a.flags == 0 and b.flags == 0 and c.flags == 0
        assert a.counts == b.counts == c.counts
