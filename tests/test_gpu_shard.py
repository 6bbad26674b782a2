"""One count shared out over two processes on the GPU (both on cuda:0: no
kernel of one waits on the other; the exchange is host-side, gloo): the
residues split by primes and rebuilt by the host CRT, and the slices of a
sliced network split by slice and summed on the host.  Both against the
oracle's exact count."""
import datetime
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

import oracle
from paper_1805_00475_gb300 import instances as I

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_1805_00475_gb300 import build as tnc_build
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import shard
    from paper_1805_00475_gb300 import slicing as S
    from paper_1805_00475_gb300 import tnc
    tnc_build.build()
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    f = I.cubic_vertex_cover(70, 1)
    plan = tnc.plan_formula(f, heuristic="gn", rank_cap=28)
    res = {"residues_int64": shard.count_residue_sharded(plan, tnc.default_primes(5), rank, world),
           "residues_tc_p8": shard.count_residue_sharded(plan, tnc.default_primes(12, "tc_p8"), rank, world,
                                                         path="tc_p8")}
    plans, _ = S.sliced_plans(f, 3)
    res["slices_int64"] = shard.count_slice_sharded(plans, tnc.default_primes(4), rank, world)
    out[rank] = res
    dist.destroy_process_group()


def test_two_processes_share_one_count():
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
        res = dict(out)
    exact = oracle.count(I.cubic_vertex_cover(70, 1), max_rank=28)
    for r in range(2):
        for key, (counts, flags) in res[r].items():
            assert flags == 0 and counts == exact, (r, key, counts, exact)
