"""Injected failures on the GPU path (no device fault is made): a
contraction whose device status is made to read as a timed-out wait reports
TNC_ERR_TIMEOUT after its work has completed, an injected launch failure
enqueues nothing, and the next calls on the same context give exact counts.
The device-side bounded waits themselves are not driven to time out on the
GPU (every wait in the tensor-core kernels waits on an outstanding TMA copy
or MMA)."""
import pytest

import oracle
from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()
    yield
    tnc.inject_failure("none")


@pytest.mark.parametrize("path", ["int64", "tc", "tc_p8"])
def test_timeout_status_is_reported_and_the_context_stays_usable(path):
    f = I.cubic_vertex_cover(70, 0)
    p = tnc.plan_formula(f, heuristic="greedy", rank_cap=28)
    R = 12 if path == "tc_p8" else 4
    tnc.inject_failure("timeout")
    with pytest.raises(tnc.TncError) as e:
        tnc.contract(p, n_residues=R, path=path)
    assert e.value.code == -5
    assert tnc.contract(p, n_residues=R, path=path).counts == oracle.count(f, max_rank=28)


def test_launch_failure_then_batch_and_noalloc_still_work():
    forms = [I.cubic_vertex_cover(40, s) for s in range(6)]
    plans = tnc.plan_many(forms, heuristic="gn")
    b = tnc.Batch(plans, n_residues=2)
    import torch
    ws = torch.empty(b.workspace_bytes(), dtype=torch.uint8, device="cuda")
    st = torch.cuda.Stream()
    b.upload(ws, st)
    tnc.inject_failure("launch")
    with pytest.raises(tnc.TncError) as e:
        b.launch(ws, st)
    assert e.value.code == -3
    b.launch(ws, st)
    assert [o.counts for o in b.download(ws, st)] == [oracle.count(f) for f in forms]
    tnc.inject_failure("launch")
    with pytest.raises(tnc.TncError):
        tnc.contract_noalloc(plans[0], n_residues=2)
    assert tnc.contract_noalloc(plans[0], n_residues=2).counts == oracle.count(forms[0])
