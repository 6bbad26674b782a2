"""Pure-Python twin of the oracle, for tiny cases -- TEST INFRASTRUCTURE.

Independent of tnc_oracle.c (no shared code) and of the product path.  Tensors
are dicts {index tuple: Python int}; counts are exact at any size.

  py_bruteforce -- Eq. z at beta -> infinity: sum over all 2^n assignments of
                   the product of clause values.
  py_contract   -- the network of Sec. 2.1 (COPY tensors on variables, clause
                   tensors on clauses, one bond per occurrence) contracted
                   pairwise, all shared bonds of a pair at once (Sec. 2.2), in
                   the given order or left to right.
"""
from __future__ import annotations

import itertools
from typing import Dict, List, Optional, Sequence, Tuple


def clause_value(kind: int, idx: Tuple[int, ...], table=None) -> int:
    """Eq. 1in3 (exactly one 1), Eq. or (not all 0), NAND (not all 1), table."""
    s = sum(idx)
    if kind == 0:
        return 1 if s == 1 else 0
    if kind == 1:
        return 1 if s > 0 else 0
    if kind == 2:
        return 1 if s < len(idx) else 0
    if kind == 3:
        j = sum(b << i for i, b in enumerate(idx))
        return int(table[j])
    raise ValueError(kind)


def py_bruteforce(f) -> List[int]:
    n_open = len(f.open_vars)
    out = [0] * (1 << n_open)
    for x in range(1 << f.n_vars):
        w = 1
        for c, k, t in zip(f.clauses, f.kinds, f.tables):
            w *= clause_value(k, tuple((x >> v) & 1 for v in c), t)
            if w == 0:
                break
        if w:
            j = sum(((x >> v) & 1) << i for i, v in enumerate(f.open_vars))
            out[j] += w
    return out


class _T:
    def __init__(self, bonds: List[int], data: Dict[Tuple[int, ...], int]):
        self.bonds = bonds
        self.data = data


def _network(f) -> Tuple[List[_T], int]:
    tensors: List[_T] = []
    occ: Dict[int, List[int]] = {v: [] for v in range(f.n_vars)}
    b = 0
    for c, k, t in zip(f.clauses, f.kinds, f.tables):
        bonds = list(range(b, b + len(c)))
        data = {}
        for idx in itertools.product((0, 1), repeat=len(c)):
            val = clause_value(k, idx, t)
            if val:
                data[idx] = val
        tensors.append(_T(bonds, data))
        for j, v in enumerate(c):
            occ[v].append(b + j)
        b += len(c)
    open_b0 = b
    for v in range(f.n_vars):
        bonds = list(occ[v])
        if v in f.open_vars:
            bonds.append(open_b0 + f.open_vars.index(v))
        r = len(bonds)
        if r == 0:
            data = {(): 2}
        else:
            data = {(0,) * r: 1, (1,) * r: 1}
        tensors.append(_T(bonds, data))
    return tensors, open_b0


def _pair(a: _T, b: _T) -> _T:
    shared = [x for x in a.bonds if x in b.bonds]
    out_bonds = [x for x in a.bonds if x not in shared] + [x for x in b.bonds if x not in shared]
    res: Dict[Tuple[int, ...], int] = {}
    for ia, va in a.data.items():
        ma = dict(zip(a.bonds, ia))
        for ib, vb in b.data.items():
            mb = dict(zip(b.bonds, ib))
            if any(ma[s] != mb[s] for s in shared):
                continue
            merged = {**ma, **mb}
            key = tuple(merged[x] for x in out_bonds)
            res[key] = res.get(key, 0) + va * vb
    return _T(out_bonds, res)


def py_contract(f, order: Optional[Sequence[Tuple[int, int]]] = None) -> List[int]:
    tensors, open_b0 = _network(f)
    live = {i: t for i, t in enumerate(tensors)}
    nxt = len(tensors)
    for a, b in (order or []):
        live[nxt] = _pair(live.pop(a), live.pop(b))
        nxt += 1
    while len(live) > 1:
        ids = sorted(live)
        a, b = ids[0], ids[1]
        live[nxt] = _pair(live.pop(a), live.pop(b))
        nxt += 1
    n_open = len(f.open_vars)
    out = [0] * (1 << n_open)
    if not live:
        out[0] = 1
        return out
    root = next(iter(live.values()))
    for idx, v in root.data.items():
        j = 0
        for ax, bond in enumerate(root.bonds):
            j |= idx[ax] << (bond - open_b0)
        out[j] += v
    return out
