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

Host-side preprocessing only (formula -> sliced formulas, choice of the
variables); every contraction runs in libtnc.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Sequence, Tuple

from . import instances as I
from . import tnc


def _clause_entry(kind: int, arity: int, idx: int, table) -> int:
    """Entry idx of a clause tensor (bit i = value of the clause's i-th
    variable): exactly-one (Eq. 1in3), OR (Eq. or), NAND, or the table."""
    if kind == I.KIND_1IN3:
        return 1 if bin(idx).count("1") == 1 else 0
    if kind == I.KIND_OR:
        return 1 if idx != 0 else 0
    if kind == I.KIND_NAND:
        return 1 if idx != (1 << arity) - 1 else 0
    return int(table[idx])


def slice_formula(f: I.Formula, fixed: Dict[int, int]) -> I.Formula:
    """The formula with the variables of `fixed` set to their values: they are
    removed (the others renumbered in order) and every clause on them becomes
    a TABLE clause over its remaining variables.  Open variables cannot be
    fixed."""
    if any(v in f.open_vars for v in fixed):
        raise ValueError("open variables cannot be sliced")
    keep = [v for v in range(f.n_vars) if v not in fixed]
    new_id = {v: i for i, v in enumerate(keep)}
    clauses, kinds, tables = [], [], []
    for c, k, t in zip(f.clauses, f.kinds, f.tables):
        if not any(v in fixed for v in c):
            clauses.append(tuple(new_id[v] for v in c))
            kinds.append(k)
            tables.append(t)
            continue
        free = [i for i, v in enumerate(c) if v not in fixed]
        base = sum(fixed[v] << i for i, v in enumerate(c) if v in fixed)
        tab = []
        for j in range(1 << len(free)):
            idx = base | sum(((j >> b) & 1) << i for b, i in enumerate(free))
            tab.append(_clause_entry(k, len(c), idx, t))
        clauses.append(tuple(new_id[c[i]] for i in free))
        kinds.append(I.KIND_TABLE)
        tables.append(tab)
    return I.Formula(len(keep), clauses, kinds, tables=tables, open_vars=[new_id[v] for v in f.open_vars],
                     name=f"{f.name}_sliced{len(fixed)}")


def _tensor_bonds(f: I.Formula, plan: tnc.Plan) -> List[set]:
    """Bonds (clause, position) of every intermediate tensor of the plan."""
    bonds: Dict[int, set] = {}
    for ci, c in enumerate(f.clauses):
        for j, v in enumerate(c):
            bonds.setdefault(ci, set()).add((ci, j))
            bonds.setdefault(f.n_cons + v, set()).add((ci, j))
    nxt, out = f.n_cons + f.n_vars, []
    for a, b in plan.steps():
        A, B = bonds.pop(a, set()), bonds.pop(b, set())
        bonds[nxt] = A ^ B
        out.append(bonds[nxt])
        nxt += 1
    return out


def choose_slice_vars(f: I.Formula, s: int, heuristic: str = "best", rank_cap: int = 64) -> List[int]:
    """s variables to fix, one at a time: the variable with the most bonds on
    the largest tensor of the current best plan (ties: most occurrences, then
    lowest index), re-planning after each choice."""
    chosen: List[int] = []
    occurrences = [0] * f.n_vars
    for c in f.clauses:
        for v in c:
            occurrences[v] += 1
    for _ in range(s):
        fixed = {v: 0 for v in chosen}
        g = slice_formula(f, fixed)
        keep = [v for v in range(f.n_vars) if v not in fixed]
        plan = tnc.plan_formula(g, heuristic=heuristic, rank_cap=rank_cap)
        tensors = _tensor_bonds(g, plan)
        if not tensors:
            break
        biggest = max(tensors, key=len)
        score: Dict[int, int] = {}
        for ci, j in biggest:
            v = keep[g.clauses[ci][j]]
            if v not in f.open_vars:
                score[v] = score.get(v, 0) + 1
        if not score:
            break
        chosen.append(min(score, key=lambda v: (-score[v], -occurrences[v], v)))
    return chosen


def sliced_plans(f: I.Formula, vars_: Sequence[int], heuristic: str = "best", rank_cap: int = 64
                 ) -> Tuple[List[tnc.Plan], List[I.Formula]]:
    """The 2^s slices of f over vars_ and their plans (planned in parallel)."""
    forms = [slice_formula(f, dict(zip(vars_, bits))) for bits in itertools.product((0, 1), repeat=len(vars_))]
    return tnc.plan_many(forms, heuristic=heuristic, rank_cap=rank_cap), forms


def count_sliced(f: I.Formula, s: int, n_residues: int = 4, path: str = "int64", heuristic: str = "best",
                 rank_cap: int = 64, primes=None, workspace=None, stream=None):
    """Exact count of f as the sum of 2^s slices (tnc_contract_sliced);
    returns (Count, the fixed variables, the slices' plans)."""
    vars_ = choose_slice_vars(f, s, heuristic, rank_cap)
    plans, _ = sliced_plans(f, vars_, heuristic, rank_cap)
    return tnc.contract_sliced(plans, n_residues=n_residues, primes=primes, workspace=workspace, stream=stream,
                               path=path), vars_, plans
