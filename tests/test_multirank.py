"""The multi-GPU path of bench.py on CPU ranks (gloo, world size 2): formula
shards are disjoint and cover the job, every rank counts its own shard with
no data exchange, and the reported time is the slowest rank's.  The host
oracle stands in for the device work here."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, batch, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import time

    import torch.distributed as dist

    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t0 = time.perf_counter()
    counts = [oracle.count(f)[0] for f in bench.workload(rank, batch)]
    mine = time.perf_counter() - t0 + 0.05 * rank  # make the ranks' times differ
    slowest = bench.max_over_ranks(mine, dist)
    out[rank] = (list(bench.shard_seeds(rank, batch)), counts, mine, slowest)
    dist.destroy_process_group()


def test_two_ranks_shard_and_take_the_slowest_time():
    import oracle
    from paper_1805_00475_gb300 import instances as I
    world, batch = 2, 3
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(world, _free_port(), batch, out), nprocs=world, join=True)
        res = dict(out)
    seeds = [s for r in range(world) for s in res[r][0]]
    assert seeds == list(range(world * batch))  # disjoint, contiguous, covering
    slowest = max(res[r][2] for r in range(world))
    assert all(abs(res[r][3] - slowest) < 1e-12 for r in range(world))
    # every rank's counts are those of its own formulas: nothing crossed ranks
    for r in range(world):
        for s, c in zip(res[r][0], res[r][1]):
            assert c == oracle.count(I.cubic_vertex_cover(60, s))[0]
