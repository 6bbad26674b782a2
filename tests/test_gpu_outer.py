"""Two shapes of the pairwise step (Sec. 2.1) with kernels of their own.

Big steps with one small operand (a skinny matrix times a tall one) run as
outer_kernel: the small operand (at most 16 free rows, at
most 8 shared values) staged in shared memory, one row of the large operand
per thread.  The formula below (#Cubic-Vertex-Cover, 100 vertices, seed 21,
bisection plan, rank 20) has such a step with 2^16 or more outputs; its count
is checked against the CPU oracle on the int64 path, the limb tensor-core
path and the 8-bit-prime path, residue by residue, and the library's launch
record shows that the kernel ran."""
import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()


@pytest.mark.parametrize("path,R", [("int64", 4), ("int64", 3), ("tc", 4), ("tc_p8", 12), ("tc_p8", 13)])
def test_outer_steps_match_oracle(path, R):
    f = I.cubic_vertex_cover(100, 21)
    p = tnc.plan_formula(f, heuristic="bisect", rank_cap=24)
    exact = oracle.count(f, max_rank=24)
    r = tnc.contract(p, n_residues=R, path=path)
    lc = tnc.last_launch_counts()
    assert lc["outer"] >= 1 and lc["level"] >= 1 and lc["leaf_fill"] >= 1
    if path == "int64":  # the plan's other big steps on the grid-wide step kernel
        assert lc["grid_step"] >= 1
    assert [int(x) for x in r.residues[0]] == [exact[0] % q for q in r.primes]
    assert r.flags == 0 and r.counts == exact


@pytest.mark.parametrize("path,R", [("tc_p8", 12), ("tc_p8", 13), ("int64", 3)])
def test_long_dot_product_matches_oracle(path, R):
    """A final step that is a dot product of two rank-20 tensors (no free
    bits, 2^20 shared values) runs split over K; on byte residues its slices
    load 4 entries at a time and add 4 products per residue per dp4a."""
    f = I.cubic_vertex_cover(100, 2)
    p = tnc.plan_formula(f, heuristic="bisect", rank_cap=24)
    exact = oracle.count(f, max_rank=24)
    r = tnc.contract(p, n_residues=R, path=path)
    assert tnc.last_launch_counts()["splitk"] >= 1
    assert [int(x) for x in r.residues[0]] == [exact[0] % q for q in r.primes]
    assert r.flags == 0 and r.counts == exact
