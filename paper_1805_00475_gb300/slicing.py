"""Bond slicing: count a formula as the sum of the counts of its slices.

Fixing variable v to 0 and to 1 splits the full trace of the network
(Sec. 2.1, Eq. z) into two traces: the variable's COPY tensor disappears and
every clause tensor on one of its bonds loses that bond (restricted to the
fixed value), so no tensor of either slice is larger than before, and the
planner can often find an order of lower rank for the smaller network.  The
memory of the contraction, which the paper names as the method's bottleneck
(Sec. 4), then shrinks by up to 2^s for s fixed variables, at the price of
2^s contractions.  Counts stay exact: the library adds the slices' residues
on the device and runs one CRT (tnc_contract_sliced).

Marshalling only: the restriction of the clause tensors, the choice of the
variables and the plans of the slices are libtnc's (tnc_slice_network,
tnc_plan_sliced); the contractions run in its kernels.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

from . import tnc


def slice_formula(f, fixed: Dict[int, int]):
    """The formula of the slice with the variables of `fixed` set to their
    values (tnc_slice_network): they leave, the others are renumbered in
    order, and every clause on them becomes a TABLE clause over its remaining
    variables.  Open variables cannot be fixed (ValueError)."""
    if any(v in f.open_vars for v in fixed):
        raise ValueError("open variables cannot be sliced")
    return tnc.slice_network(f, fixed)


def choose_slice_vars(f, s: int, heuristic: str = "best", rank_cap: int = 64) -> List[int]:
    """The s variables tnc_plan_sliced fixes (cost-checked, one at a time)."""
    return tnc.plan_sliced(f, s, heuristic=heuristic, rank_cap=rank_cap)[1]


def sliced_plans(f, s: int, heuristic: str = "best", rank_cap: int = 64) -> Tuple[List[tnc.Plan], List[int]]:
    """The plans of the 2^s slices of f and the fixed variables (tnc_plan_sliced)."""
    return tnc.plan_sliced(f, s, heuristic=heuristic, rank_cap=rank_cap)


def count_sliced(f, s: int, n_residues: int = 4, path: str = "int64", heuristic: str = "best",
                 rank_cap: int = 64, primes=None, workspace=None, stream=None):
    """Exact count of f as the sum of 2^s slices (tnc_plan_sliced +
    tnc_contract_sliced); returns (Count, the fixed variables, the slices' plans)."""
    plans, vars_ = tnc.plan_sliced(f, s, heuristic=heuristic, rank_cap=rank_cap)
    return tnc.contract_sliced(plans, n_residues=n_residues, primes=primes, workspace=workspace, stream=stream,
                               path=path), vars_, plans
