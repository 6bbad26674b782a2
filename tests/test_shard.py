"""Sharding one count over processes (host side, CPU ranks on gloo).

The combine is libtnc's host code (tnc_crt_host, tnc_residue_add_host) and
the slices are libtnc's (tnc_slice_network); the device contraction of each
rank's share is stood in for by the oracle's exact count reduced modulo the
rank's primes (the GPU form of the same runs is tests/test_gpu_shard.py).
Also: a rank that never reaches the gather makes the others fail with an
error within the process group's timeout, instead of hanging."""
import datetime
import itertools
import os
import random
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import shard
from paper_1805_00475_gb300 import slicing as S
from paper_1805_00475_gb300 import tnc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_crt_host_is_the_chinese_remainder():
    """Values below the product of the primes come back exactly, for 30-bit
    primes, 8-bit primes and a mix in any order (the CRT's uniqueness)."""
    rng = random.Random(1)
    for primes in (tnc.default_primes(5), tnc.default_primes(20, "tc_p8"),
                   [251, 1073741789, 3, 2147483647, 199]):
        M = 1
        for p in primes:
            M *= p
        xs = [0, 1, M - 1] + [rng.randrange(M) for _ in range(20)]
        res = [[x % p for p in primes] for x in xs]
        assert tnc.crt_host(primes, res) == xs


def test_residue_add_host_is_modular_addition():
    primes = [1073741789, 251, 7]
    rng = np.random.default_rng(2)
    a = np.stack([rng.integers(0, p, 50) for p in primes], axis=1).astype(np.uint32)
    b = np.stack([rng.integers(0, p, 50) for p in primes], axis=1).astype(np.uint32)
    want = (a.astype(np.int64) + b) % np.array(primes)
    assert (tnc.residue_add_host(primes, a.copy(), b) == want).all()


def _rank_residues(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import shard
    from paper_1805_00475_gb300 import tnc
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    f = I.cubic_vertex_cover(60, 3)
    f.open_vars = [0, 7]
    primes = tnc.default_primes(5)
    mine = shard.split_round_robin(primes, rank, world)
    exact = oracle.count(f)  # stands in for tnc.contract(plan, primes=mine)
    res = np.array([[c % p for p in mine] for c in exact], dtype=np.uint32)
    parts = shard._gather((mine, res), world)
    plan = tnc.plan_formula(f, heuristic="gn")
    out[rank] = shard.combine_residue_shards(parts, plan.stats.log2_bound)
    dist.destroy_process_group()


def test_two_ranks_residue_shards_rebuild_the_count():
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_residues, args=(2, _free_port(), out), nprocs=2, join=True)
        res = dict(out)
    f = I.cubic_vertex_cover(60, 3)
    f.open_vars = [0, 7]
    exact = oracle.count(f)
    for r in range(2):
        counts, flags = res[r]
        assert flags == 0 and counts == exact


def _rank_slices(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import oracle
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import shard
    from paper_1805_00475_gb300 import slicing as S
    from paper_1805_00475_gb300 import tnc
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=60))
    f = I.one_in_three(22, 14, 4)
    vs = S.choose_slice_vars(f, 3)
    primes = tnc.default_primes(2)
    slices = [dict(zip(vs, bits)) for bits in itertools.product((0, 1), repeat=3)]
    acc = None
    for fixed in shard.split_round_robin(slices, rank, world):
        c = oracle.count(S.slice_formula(f, fixed))  # stands in for the device contraction of the slice
        res = np.array([[x % p for p in primes] for x in c], dtype=np.uint32)
        acc = res if acc is None else tnc.residue_add_host(primes, acc, res)
    parts = shard._gather(acc, world)
    out[rank] = shard.combine_slice_shards(parts, primes, None)
    dist.destroy_process_group()


def test_three_ranks_slice_shards_sum_to_the_count():
    """8 slices over 3 ranks (uneven shares); the host sums and remainders."""
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_slices, args=(3, _free_port(), out), nprocs=3, join=True)
        res = dict(out)
    exact = oracle.count(I.one_in_three(22, 14, 4))
    for r in range(3):
        assert res[r][0] == exact


def _rank_lost(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_1805_00475_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=3))
    if rank == 1:
        out[rank] = "left before the gather"
        return  # this rank's shard is lost: it never joins the exchange
    try:
        shard._gather(np.zeros((1, 2), dtype=np.uint32), world)
        out[rank] = "gathered"
    except Exception as e:  # gloo reports the missing peer within the timeout
        out[rank] = "error: " + type(e).__name__


def test_a_lost_shard_is_an_error_not_a_hang():
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        ctx = mp.spawn(_rank_lost, args=(2, _free_port(), out), nprocs=2, join=False)
        assert ctx.join(timeout=60) or ctx.join(timeout=60)
        res = dict(out)
    assert res[1] == "left before the gather"
    assert res[0].startswith("error"), res[0]
