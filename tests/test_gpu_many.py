"""tnc_contract_many: independent formulas contracted with their tree levels
merged (one launch per level for the small steps of every formula of a
group).  Every residue and CRT value against the oracle, on every path, for
groups of one formula up to all of them, with open variables, weighted
tables, an empty network and uneven sizes; and sliced counts whose slices run
merged when the workspace holds several."""
import random

import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import slicing as S
from paper_1805_00475_gb300 import tnc
from _util import random_formula

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


def _formulas():
    rng = random.Random(7)
    fs = [I.cubic_vertex_cover(n, s) for n, s in ((20, 0), (60, 1), (70, 2), (40, 3))]
    fs += [I.one_in_three(n, int(n * 0.6), s) for n, s in ((30, 4), (50, 5), (80, 6))]
    g = I.one_in_three(40, 24, 9)
    g.open_vars = [1, 5, 7]
    fs.append(g)
    fs.append(random_formula(rng, 14, 12, n_open=2, weights=(0, 1, 3, 7)))
    fs.append(I.Formula(0, [], []))
    fs.append(I.worked_example())
    return fs


@pytest.mark.parametrize("path,R", [("int64", 4), ("tc", 3), ("tc_p8", 12)])
@pytest.mark.parametrize("group", [1, 3, 100])
def test_many_matches_oracle(path, R, group):
    fs = _formulas()
    plans = [tnc.plan_formula(f, heuristic="greedy", rank_cap=28) for f in fs]
    want = [oracle.count(f, max_rank=28) for f in fs]
    nb = tnc.workspace_bytes_many(plans, R, path, group=group)
    import torch
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    got = tnc.contract_many(plans, n_residues=R, path=path, workspace=ws)
    for f, w, r in zip(fs, want, got):
        assert r.residues.tolist() == oracle.residues(w, r.primes), f.name
        if r.flags == 0:
            assert r.counts == w, f.name
    lc = tnc.last_launch_counts()
    if group >= len(fs):  # one group: one leaf fill per residue pass for all formulas
        passes = {"int64": 1, "tc": R, "tc_p8": 3}[path]
        assert lc["leaf_fill"] == passes


def test_many_equals_one_by_one_on_c3_sizes():
    plans = [p for p in tnc.plan_many(I.batch_one_in_three(48, 2026), heuristic="best", rank_cap=64)
             if p.stats.max_rank <= 22][:24]
    one = [tnc.contract(p, n_residues=8, path="tc_p8") for p in plans]
    many = tnc.contract_many(plans, n_residues=8, path="tc_p8", group=8)
    assert [r.residues.tolist() for r in many] == [r.residues.tolist() for r in one]
    assert [r.flags for r in many] == [r.flags for r in one]


def test_many_rejects_a_workspace_too_small_for_one_plan():
    import torch
    plans = [tnc.plan_formula(I.cubic_vertex_cover(60, 0))]
    ws = torch.empty(4096, dtype=torch.uint8, device="cuda")
    with pytest.raises(tnc.TncError) as e:
        tnc.contract_many(plans, n_residues=2, workspace=ws)
    assert e.value.code == -4


def test_sliced_slices_merge_in_a_large_workspace():
    import torch
    f = I.cubic_vertex_cover(70, 2)
    plans, _ = S.sliced_plans(f, 3)
    want = oracle.count(f, max_rank=28)
    small = tnc.contract_sliced(plans, n_residues=3)
    levels_small = tnc.last_launch_counts()["leaf_fill"]
    nb = tnc.workspace_bytes_many(plans, 3, group=8) + (1 << 20)
    big = tnc.contract_sliced(plans, n_residues=3, workspace=torch.empty(nb, dtype=torch.uint8, device="cuda"))
    assert small.counts == big.counts == want
    assert tnc.last_launch_counts()["leaf_fill"] < levels_small  # merged: fewer leaf fills than slices
