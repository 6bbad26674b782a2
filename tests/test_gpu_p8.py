"""The 8-bit-prime tensor-core path (TNC_PATH_TC_P8): residues modulo primes
<= 251, one fp16 limb each, dense steps as TMA-fed tcgen05 GEMMs with the fp32
accumulator reduced in place every 1024 shared values.  Residues are compared
with the CPU oracle's exact count reduced mod each prime, and the CRT values
with the oracle (small cases) or with the int64 path (large cases)."""
import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


ORACLE_CASES = [(70, "greedy", 0), (70, "greedy", 1), (70, "greedy", 2), (70, "gn", 1), (70, "bisect", 0),
                (70, "bisect", 1), (80, "greedy", 0), (80, "gn", 2), (80, "bisect", 2)]


@pytest.mark.parametrize("n,h,seed", ORACLE_CASES)
def test_p8_matches_oracle(n, h, seed):
    f = I.cubic_vertex_cover(n, seed)
    p = tnc.plan_formula(f, heuristic=h, rank_cap=28)
    exact = oracle.count(f, max_rank=28)
    r = tnc.contract(p, n_residues=12, path="tc_p8")
    assert tnc.last_launch_counts()["p8_gemm"] >= 1
    assert [int(x) for x in r.residues[0]] == [exact[0] % q for q in r.primes]
    assert r.flags == 0 and r.counts == exact


def test_p8_oracle_cases_cover_every_tile_width_and_both_orientations():
    """The oracle cases above, by the library's own launch record: the narrow
    tile widths that steps with less than a wave of tiles take (64, 128 and
    256: tests/test_gpu_dense_branches.py), rows from A and from B,
    zero-padded and unpadded shared dimensions."""
    widths, swapped, unswapped, padded, unpadded = set(), 0, 0, 0, 0
    for n, h, seed in ORACLE_CASES:
        p = tnc.plan_formula(I.cubic_vertex_cover(n, seed), heuristic=h, rank_cap=28)
        tnc.contract(p, n_residues=4, path="tc_p8")
        lc = tnc.last_launch_counts()
        widths |= {w for w, c in lc["p8_tile_n"].items() if c}
        swapped += lc["p8_swapped"]
        unswapped += lc["p8_gemm"] - lc["p8_swapped"]
        padded += lc["p8_padded"]
        unpadded += lc["p8_gemm"] - lc["p8_padded"]
    assert {16, 32} <= widths
    assert swapped and unswapped and padded and unpadded


@pytest.mark.parametrize("n,h,seed", [(100, "greedy", 0), (100, "greedy", 2), (120, "greedy", 2), (120, "bisect", 2)])
def test_p8_matches_int64_with_k_split(n, h, seed):
    f = I.cubic_vertex_cover(n, seed)
    p = tnc.plan_formula(f, heuristic=h, rank_cap=30)
    a = tnc.contract(p, n_residues=5, path="int64")
    b = tnc.contract(p, n_residues=20, path="tc_p8")
    assert tnc.last_launch_counts()["p8_gemm"] >= 1
    assert a.flags == 0 and b.flags == 0
    assert a.counts == b.counts


def test_p8_k_split_cases_really_split():
    splits = 0
    for n, h, seed in [(100, "greedy", 2), (120, "greedy", 2)]:
        p = tnc.plan_formula(I.cubic_vertex_cover(n, seed), heuristic=h, rank_cap=30)
        tnc.contract(p, n_residues=4, path="tc_p8")
        splits += tnc.last_launch_counts()["p8_split"]
    assert splits >= 2


def test_p8_many_chunks_match_int64():
    """A dense step with 2^16 shared values (256 x 256 tiles on CTA pairs)
    over 2^4 K slices: 4 chunks of 1024 per tile, each reduced in place in
    TMEM before the next."""
    f = I.cubic_vertex_cover(180, 1)
    p = tnc.plan_formula(f, heuristic="best", rank_cap=30)
    a = tnc.contract(p, n_residues=7, path="int64")
    b = tnc.contract(p, n_residues=26, path="tc_p8")
    assert tnc.last_launch_counts()["p8_max_chunks"] >= 4
    assert a.flags == 0 and b.flags == 0
    assert a.counts == b.counts


def test_p8_wide_tiles_match_int64():
    """Steps with at least 456 tiles of 128 x 256 run 256-wide tiles: two
    residues per round in TMEM, each round writing its two bytes of every
    entry.  Counts equal the int64 path's (disjoint primes, both CRTs)."""
    f = I.cubic_vertex_cover(180, 1)
    p = tnc.plan_formula(f, heuristic="best", rank_cap=30)
    a = tnc.contract(p, n_residues=7, path="int64")
    for R in (26, 21):  # 4-residue passes and a last pass of 2 residues; then of 1 residue
        b = tnc.contract(p, n_residues=R, path="tc_p8")
        assert tnc.last_launch_counts()["p8_tile_n"][256] >= 1
        assert a.flags == 0 and b.flags == 0
        assert a.counts == b.counts


def test_p8_one_in_three_with_open_bonds():
    f = I.one_in_three(60, 40, 3)
    f.open_vars = [0, 5, 9]
    p = tnc.plan_formula(f, heuristic="greedy", rank_cap=28)
    exact = oracle.count(f, max_rank=28)
    r = tnc.contract(p, n_residues=10, path="tc_p8")
    assert r.counts == exact
    for e, row in zip(exact, r.residues):
        assert [int(x) for x in row] == [e % q for q in r.primes]


def test_p8_smallest_primes():
    """p = 3 (residues -1, 0, 1) up to 251, given by the caller."""
    f = I.cubic_vertex_cover(70, 1)
    p = tnc.plan_formula(f, heuristic="greedy", rank_cap=28)
    primes = [3, 5, 7, 11, 13, 127, 251]
    exact = oracle.count(f, max_rank=28)[0]
    r = tnc.contract(p, n_residues=len(primes), primes=primes, path="tc_p8")
    assert [int(x) for x in r.residues[0]] == [exact % q for q in primes]


def test_p8_rejects_bad_options():
    f = I.cubic_vertex_cover(20, 0)
    p = tnc.plan_formula(f)
    with pytest.raises(tnc.TncError):
        tnc.contract(p, n_residues=2, primes=[257, 251], path="tc_p8")
    with pytest.raises(tnc.TncError):
        tnc.contract(p, n_residues=2, primes=[1073741789, 251], path="tc_p8")
    with pytest.raises(tnc.TncError):
        tnc.contract(p, n_residues=2, primes=[251, 251], path="tc_p8")
    with pytest.raises(tnc.TncError):
        tnc.Batch([p], n_residues=4, path="tc_p8")
