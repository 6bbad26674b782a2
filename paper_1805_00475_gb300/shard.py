"""Counting one formula on several processes, one GPU each (torch.distributed
for the host-side exchange; no device collective).

Two ways to share out one count (the paper leaves distributed contraction as
a prospect, Sec. 4):

  * residues: the primes are split over the ranks (each residue is an
    independent contraction); every rank contracts the whole network modulo
    its own primes; the residue arrays are gathered and every rank rebuilds
    the exact count by the CRT on the host (tnc_crt_host);
  * slices: the 2^s slices of a sliced network (tnc_plan_sliced) are split
    over the ranks; every rank adds its slices' residues on its device
    (tnc_contract_sliced); the per-rank sums are gathered, added modulo the
    primes on the host (tnc_residue_add_host) and remaindered (tnc_crt_host).

Marshalling only: every contraction and every combine is libtnc's.  The
gather is `all_gather_object` of small numpy arrays (gloo or NCCL).
"""
from __future__ import annotations

from typing import List, Optional, Sequence

import numpy as np

from . import tnc


def split_round_robin(items: Sequence, rank: int, world: int) -> list:
    """Rank r's share: items r, r + world, r + 2 world, ..."""
    return list(items)[rank::world]


def _gather(obj, world: int, group=None):
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, obj, group=group)
    return out


def certified(log2_bound: float, primes: Sequence[int]) -> bool:
    """The exact count is below the product of the primes (see TNC_MAYBE_WRAPPED)."""
    return log2_bound < float(np.sum(np.log2(np.asarray(primes, dtype=np.float64)))) - 1e-9


def count_residue_sharded(plan: tnc.Plan, primes: Sequence[int], rank: int, world: int, path: str = "int64",
                          group=None, stream=None):
    """Exact counts of `plan` with the primes shared out over the ranks.
    Returns (counts, flags): flags = TNC_MAYBE_WRAPPED when the bound is not
    certified by the product of all primes."""
    mine = split_round_robin(primes, rank, world)
    res = tnc.contract(plan, n_residues=len(mine), primes=mine, path=path, stream=stream).residues if mine else None
    parts = _gather((mine, None if res is None else np.asarray(res, dtype=np.uint32)), world, group)
    return combine_residue_shards(parts, plan.stats.log2_bound)


def combine_residue_shards(parts, log2_bound: float):
    """parts: per rank (its primes, residues [n_out, len(primes)] or None).
    Interleaves the columns back into one [n_out, R] array and remainders."""
    primes = [p for pr, _ in parts for p in pr]
    cols = [res for _, res in parts if res is not None]
    res = np.concatenate(cols, axis=1) if cols else np.zeros((1, 0), dtype=np.uint32)
    counts = tnc.crt_host(primes, res)
    return counts, 0 if certified(log2_bound, primes) else tnc.TNC_MAYBE_WRAPPED


def count_slice_sharded(plans: List[tnc.Plan], primes: Sequence[int], rank: int, world: int,
                        path: str = "int64", group=None, stream=None):
    """Exact counts of the sum of the slices' counts with the slices shared out
    over the ranks.  Returns (counts, flags)."""
    mine = split_round_robin(plans, rank, world)
    res = None
    if mine:
        r = tnc.contract_sliced(mine, n_residues=len(primes), primes=list(primes), path=path, stream=stream)
        res = np.asarray(r.residues, dtype=np.uint32)
    parts = _gather(res, world, group)
    bound = None
    for p in plans:  # log2 of the sum of the slices' bounds
        b = p.stats.log2_bound
        bound = b if bound is None else max(bound, b) + float(np.log2(1.0 + 2.0 ** -abs(bound - b)))
    return combine_slice_shards(parts, primes, bound)


def combine_slice_shards(parts, primes: Sequence[int], log2_bound: Optional[float]):
    """parts: per rank its slices' residue sum [n_out, R] (or None)."""
    acc = None
    for res in parts:
        if res is None:
            continue
        if acc is None:
            acc = np.array(res, dtype=np.uint32, copy=True)
        else:
            tnc.residue_add_host(primes, acc, res)
    counts = tnc.crt_host(primes, acc)
    return counts, 0 if log2_bound is None or certified(log2_bound, primes) else tnc.TNC_MAYBE_WRAPPED
