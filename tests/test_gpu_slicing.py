"""Bond slicing on the GPU (tnc_contract_sliced): the slices' residues are
added on the device and one CRT gives the count, equal to the oracle's (small
networks) and to the unsliced contraction (a rank-29 network)."""
import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import slicing as S
from paper_1805_00475_gb300 import tnc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


@pytest.mark.parametrize("s", [1, 2, 3])
@pytest.mark.parametrize("path,R", [("int64", 3), ("tc", 3), ("tc_p8", 12)])
def test_sliced_count_matches_oracle(s, path, R):
    f = I.cubic_vertex_cover(70, 2)
    exact = oracle.count(f, max_rank=28)
    r, vs, plans = S.count_sliced(f, s, n_residues=R, path=path)
    assert len(plans) == 2 ** s and len(vs) == s
    assert r.counts == exact and r.flags == 0


def test_sliced_open_bonds_match_oracle():
    f = I.one_in_three(60, 40, 5)
    f.open_vars = [1, 8]
    r, _, _ = S.count_sliced(f, 2, n_residues=3)
    assert r.counts == oracle.count(f, max_rank=28)


def test_sliced_rank29_network_matches_unsliced():
    f = I.cubic_vertex_cover(180, 3)
    whole = tnc.contract(tnc.plan_formula(f, heuristic="best", rank_cap=30), n_residues=20, path="tc_p8")
    r, vs, plans = S.count_sliced(f, 3, n_residues=20, path="tc_p8")
    assert max(p.stats.max_rank for p in plans) <= 27
    assert whole.flags == 0 and r.flags == 0
    assert r.counts == whole.counts
