"""Host-side fault injection (tnc_inject_failure) and the library's handling
of the failures it makes: error codes and messages, all-or-nothing cleanup of
tnc_plan_many, and a usable library afterwards.  No device is touched: the
LAUNCH injection fires before a contraction's first device call.  Also the
scorer parameter files (tnc_learned_save / tnc_learned_load)."""
import ctypes
import os

import numpy as np
import pytest

from paper_1805_00475_gb300 import build as tnc_build
from paper_1805_00475_gb300 import instances as I
from paper_1805_00475_gb300 import tnc


@pytest.fixture(scope="module", autouse=True)
def built():
    tnc_build.build()
    yield
    tnc.inject_failure("none")


def test_injected_allocation_failure_in_build_and_plan():
    f = I.cubic_vertex_cover(20, 0)
    tnc.inject_failure("nomem")
    with pytest.raises(tnc.TncError) as e:
        tnc.build_network(f)
    assert e.value.code == -6
    net = tnc.build_network(f)  # disarmed after firing once
    tnc.inject_failure("nomem")
    with pytest.raises(tnc.TncError) as e:
        tnc.plan(net)
    assert e.value.code == -6
    assert tnc.plan(net).stats.n_steps > 0


def test_injected_plan_failure_makes_plan_many_all_or_nothing():
    forms = [I.cubic_vertex_cover(20, s) for s in range(12)]
    tnc.inject_failure("plan", after=5)
    with pytest.raises(tnc.TncError) as e:
        tnc.plan_many(forms, heuristic="greedy")
    assert e.value.code == -2 and "injected" in str(e.value) and "formula" in str(e.value)
    plans = tnc.plan_many(forms, heuristic="greedy")
    assert len(plans) == 12 and all(p.stats.n_steps > 0 for p in plans)


def test_injected_launch_failure_touches_no_device():
    """With a workspace address that is never dereferenced, the armed launch
    failure returns TNC_ERR_CUDA before any CUDA call (there is no GPU here)."""
    p = tnc.plan_formula(I.cubic_vertex_cover(20, 1), heuristic="greedy")
    o, _ = tnc._opts(2, None)
    nb = tnc.workspace_bytes(p, 2)
    res = np.zeros((1, 2), dtype=np.uint32)
    limbs = np.zeros((1, 2), dtype=np.uint32)
    c = tnc._Count(tnc._p(res, ctypes.c_uint32), tnc._p(limbs, ctypes.c_uint32), 1, 2, 0, 0, 0)
    tnc.inject_failure("launch")
    rc = tnc.lib().tnc_contract(p.h, ctypes.byref(o), ctypes.c_void_p(1 << 20), nb, None, ctypes.byref(c))
    assert rc == -3 and b"injected" in tnc.lib().tnc_last_error()


def test_injection_rejects_unknown_kinds():
    assert tnc.lib().tnc_inject_failure(9, 0) == -1
    assert tnc.lib().tnc_inject_failure(1, -1) == -1


def test_learned_parameters_round_trip_and_are_checked(tmp_path):
    params = tnc.mlp_init(3)
    path = str(tmp_path / "scorer.bin")
    tnc.learned_save(path, params)
    assert (tnc.learned_load(path) == params).all()
    raw = bytearray(open(path, "rb").read())
    raw[100] ^= 1  # one flipped bit: checksum mismatch
    bad = str(tmp_path / "bad.bin")
    open(bad, "wb").write(bytes(raw))
    with pytest.raises(tnc.TncError):
        tnc.learned_load(bad)
    open(bad, "wb").write(bytes(raw[:-9]))  # truncated
    with pytest.raises(tnc.TncError):
        tnc.learned_load(bad)
    with pytest.raises(tnc.TncError):
        tnc.learned_load(str(tmp_path / "missing.bin"))
