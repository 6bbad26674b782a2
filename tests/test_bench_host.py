"""Host logic of bench.py that decides what the JSON line reports: the DRAM
traffic of a profile summary is reported only for the kernel sources and the
planner it was captured with, and the committed summary names the current
sources and the default planner."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _profile(tmp_path, sha, planner, value=123456789):
    p = tmp_path / "prof.md"
    p.write_text(f"# x\n\ntraffic_bytes_per_launch = {value}, kernel_source_sha = {sha}, planner = {planner}\n")
    return str(p)


def test_traffic_is_reported_only_for_the_captured_sources_and_planner(tmp_path):
    sha = bench.kernel_source_sha(bench.C2_KERNEL_SOURCES)
    t, why = bench.captured_traffic(_profile(tmp_path, sha, "coarsen"), bench.C2_KERNEL_SOURCES, "coarsen")
    assert t == 123456789.0 and "ncu capture" in why
    t, why = bench.captured_traffic(_profile(tmp_path, sha, "best"), bench.C2_KERNEL_SOURCES, "coarsen")
    assert t is None and "planner" in why
    t, why = bench.captured_traffic(_profile(tmp_path, "0" * 16, "coarsen"), bench.C2_KERNEL_SOURCES, "coarsen")
    assert t is None and "kernel changed" in why
    t, why = bench.captured_traffic(str(tmp_path / "missing.md"), bench.C2_KERNEL_SOURCES, "coarsen")
    assert t is None
    p = tmp_path / "prof2.md"
    p.write_text(f"traffic_bytes_per_launch = 5, kernel_source_sha = {sha}, planner = coarsen, plan_macs = 1000\n")
    assert bench.captured_traffic(str(p), bench.C2_KERNEL_SOURCES, "coarsen", 1000.0)[0] == 5.0
    t, why = bench.captured_traffic(str(p), bench.C2_KERNEL_SOURCES, "coarsen", 999.0)
    assert t is None and "plans changed" in why


def test_committed_profile_matches_the_default_run(monkeypatch):
    """The C2 summary's key line names the current batch-kernel sources and
    bench.py's default planner, so the default line carries measured traffic."""
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    default_planner = bench.parse().planner
    t, why = bench.captured_traffic(bench.C2_PROFILE, bench.C2_KERNEL_SOURCES, default_planner)
    assert t is not None, why
    # the plans of the default workload are the captured ones (host planning only)
    from paper_1805_00475_gb300 import build as tnc_build
    from paper_1805_00475_gb300 import tnc
    tnc_build.build()
    plans = tnc.plan_many(bench.workload(0, 8192), heuristic=default_planner)
    macs = sum(p.stats.total_macs for p in plans) * bench.R
    t, why = bench.captured_traffic(bench.C2_PROFILE, bench.C2_KERNEL_SOURCES, default_planner, macs)
    assert t is not None, why
    assert 1e8 < t < 1e10
