"""Throughput of exact tensor-network model counting on GB300.

Workload (one step): a batch of B #Cubic-Vertex-Cover formulas, each on a
seeded random simple connected cubic graph with n = 60 vertices
(configuration model with rejection), counted exactly as R = 4 residues
modulo the largest primes below 2^30 plus the CRT value, on the int64
CUDA-core path, contracted along tensor-GN / bisection / greedy plans (the
cheapest per formula) in one persistent, graph-captured launch.

Metric: exact model counts per second (formulas fully counted: all residues
and the CRT) and modular MACs per second (sum over steps of 2^(a+b-k), times R).

Beside it, in the same line (block "c4"): the comparison of the arithmetic
paths on 16 #Cubic-Vertex-Cover formulas on 180 vertices (tensor-greedy-free
best plans of rank <= 30): the 8-bit-prime tensor-core path timed over the
steps, the int64 CUDA-core path and the limb tensor-core path timed once, the
same counts asserted, and the dense steps' roofline from CUDA events.

  python bench.py [--gpus N --steps K --warmup W --batch B]
  python bench.py --impl reference ...   # the CPU oracle as the reference arm

Under torchrun (N > 1) every rank counts its own B formulas (different seeds):
weak scaling, no data-path collective; value = all ranks' formulas / max time.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact model counts/s"
UNIT = "counts/s"
N_VERTS = 60
R = 4


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8192, help="formulas per rank per step")
    ap.add_argument("--impl", default="tnc", choices=["tnc", "reference"])
    ap.add_argument("--planner", default="coarsen",
                    help="c2 planner: coarsen (tensor-greedy coarsening finished by the best of the paper's "
                         "heuristics, fewest MACs) or any single heuristic")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="oracle sample budget")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c4", action="store_true", help="default run: leave out the C4 comparison block")
    ap.add_argument("--min-timed-s", type=float, default=1.0,
                    help="c2: repeat the block of K timed steps until this much device time is covered")
    ap.add_argument("--e2e-split", default="0.35,0.65",
                    help="c2 e2e: shares of the formulas in consecutive batches on their own streams, so "
                         "that one batch's upload overlaps the previous batch's kernel")
    ap.add_argument("--launch", default="", help="c2: fixed launch shape THREADS,SMEM_BYTES[,CTAS_PER_SM] instead of the autotuner")
    ap.add_argument("--config", default="c2", choices=["c2", "c3", "c4", "c5", "slicing", "fig4c", "planners"],
                    help="c2: batch of cubic VC n=60 (default); c3: 4096 uneven monotone 1-in-3 "
                         "formulas, 2 residues; c4: cubic VC n=180, 8 residues, tensor-core vs CUDA-core path")
    ap.add_argument("--formulas", type=int, default=0, help="c3/c4/c5: number of formulas (0 = the config's)")
    ap.add_argument("--c4-compare", default="tc,int64",
                    help="c4: arithmetic paths timed once beside the 8-bit-prime path ('' for none)")
    ap.add_argument("--train-formulas", type=int, default=4000, help="c5: generated training formulas")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard_seeds(rank: int, batch: int):
    """Seeds of one rank's formulas: ranks own disjoint, contiguous seed ranges
    (weak scaling: every rank counts `batch` formulas of its own)."""
    return range(rank * batch, (rank + 1) * batch)


def workload(rank: int, batch: int):
    from paper_1805_00475_gb300 import instances as I
    return [I.cubic_vertex_cover(N_VERTS, s) for s in shard_seeds(rank, batch)]


def max_over_ranks(value: float, dist, device=None) -> float:
    """The slowest rank's time: the one all-reduce of the multi-GPU run (it
    carries timings only; no formula data moves between ranks)."""
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config(args, world):
    return {"workload": f"cubic_vertex_cover_n{N_VERTS}_R{R}_batch{args.batch}",
            "formulas_per_rank": args.batch, "n_vertices": N_VERTS, "residues": R,
            "path": "int64", "planner": args.planner, "launch": "persistent, graph-captured",
            "l2": "flushed (256 MiB write) between timed steps", "world_size": world}


# --------------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for row in csv.reader(io.StringIO(out)):
            if len(row) < 9:
                continue
            try:
                sm.append(float(row[1]))
                mx.append(float(row[2]))
            except ValueError:
                continue
            for nm, v in zip(names, row[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- oracle

def oracle_sample(forms, budget_s: float):
    """Time the CPU oracle, as it stands, on formulas of the workload until the
    budget is spent; returns (formulas done, seconds, threads)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    done = 0
    for f in forms:
        oracle.count(f)
        done += 1
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return done, el, threads


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# --------------------------------------------------------------------- arms

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    forms = workload(0, min(args.batch, 4096))
    import oracle
    oracle.build()
    t = time.perf_counter()
    oracle.count(forms[0])
    one = max(time.perf_counter() - t, 1e-4)
    per_step = max(1, min(len(forms), int(2.0 / one)))
    for i in range(args.warmup):
        for f in forms[:per_step]:
            oracle.count(f)
    times = []
    for s in range(args.steps):
        t = time.perf_counter()
        for f in forms[:per_step]:
            oracle.count(f)
        times.append(time.perf_counter() - t)
    ms = 1000.0 * sum(times) / len(times)
    value = per_step / (ms / 1000.0)
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bigint", "data": "synthetic",
            "config": config(args, 1),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} formulas of the workload per step (C bigint oracle, "
                                       f"tensor-greedy order)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def c4_workload(count=16, n=180):
    """#Cubic-Vertex-Cover, n = 180: seeds from 0 upwards whose best heuristic
    plan keeps every tensor at rank <= 30."""
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import tnc
    kept = []
    s = 0
    while len(kept) < count:
        f = I.cubic_vertex_cover(n, s)
        try:
            kept.append((s, f, tnc.plan_formula(f, heuristic="best", rank_cap=30)))
        except tnc.TncError:
            pass
        s += 1
    return kept


def run_c3(args):
    """4096 monotone 1-in-3 formulas, n ~ U{50..150}, m = round(n U[0.5, 0.8)),
    every one counted on the device, from one host thread on one stream:
      * light plans (<= 2^24 MACs, rank <= 16; the descriptors of a formula fit
        in shared memory): one persistent, graph-captured, autotuned batch
        launch, 2 residues below 2^30;
      * heavy plans (re-planned by the portfolio of the paper's heuristics):
        tnc_contract_many on the 8-bit-prime tensor-core path, 8 primes <= 251
        (product 2^62.8), tree levels merged across the formulas of a group;
      * plans still above rank 26: bond-sliced (tnc_plan_sliced) to rank <= 26
        and counted by tnc_contract_sliced, same primes.
    Counts whose certified bound exceeds the product of the primes carry
    TNC_MAYBE_WRAPPED (residues exact, CRT value the count modulo that product)."""
    import torch
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import slicing as S
    from paper_1805_00475_gb300 import tnc
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    Rc, R8, n_total = 2, 8, args.formulas or 4096
    light_macs, rank_many, ws_gb = 2.0 ** 24, 26, 16
    forms = I.batch_one_in_three(n_total, 2026)
    t = time.perf_counter()
    plans = tnc.plan_many(forms, heuristic="best", rank_cap=64)
    is_light = [p.stats.total_macs <= light_macs and p.stats.max_rank <= 16 for p in plans]
    heavy_idx = [i for i, l in enumerate(is_light) if not l]
    heavy_plans = tnc.plan_many([forms[i] for i in heavy_idx], heuristic="portfolio", rank_cap=64)
    many_idx = [i for i, p in zip(heavy_idx, heavy_plans) if p.stats.max_rank <= rank_many]
    many = [p for p in heavy_plans if p.stats.max_rank <= rank_many]
    big_idx = [i for i, p in zip(heavy_idx, heavy_plans) if p.stats.max_rank > rank_many]
    sliced = []
    for i, p in zip(big_idx, [p for p in heavy_plans if p.stats.max_rank > rank_many]):
        s = 1
        while True:
            sp, vs = S.sliced_plans(forms[i], s, heuristic="best")
            if max(q.stats.max_rank for q in sp) <= rank_many or s >= 10:
                break
            s += 1
        sliced.append((i, sp, vs))
    plan_s = time.perf_counter() - t
    light = [p for p, l in zip(plans, is_light) if l]
    batch = tnc.Batch(light, n_residues=Rc)
    ws_b = torch.empty(batch.workspace_bytes(), dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    batch.upload(ws_b, stream)
    tuned = batch.autotune(ws_b, stream)
    ws = torch.empty(ws_gb << 30, dtype=torch.uint8, device=dev)
    macs_light = sum(p.stats.total_macs for p in light) * Rc
    macs_many = sum(p.stats.total_macs for p in many) * R8
    macs_sliced = sum(q.stats.total_macs for _, sp, _ in sliced for q in sp) * R8
    phase_ms = [[], [], []]
    results = {}

    def one_step():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ev[0].record(stream)
        batch.launch(ws_b, stream)
        ev[1].record(stream)
        res_many = tnc.contract_many(many, n_residues=R8, path="tc_p8", workspace=ws, stream=stream)
        ev[2].record(stream)
        res_sliced = [tnc.contract_sliced(sp, n_residues=R8, path="tc_p8", workspace=ws, stream=stream)
                      for _, sp, _ in sliced]
        ev[3].record(stream)
        res_light = batch.download_flat(ws_b, stream)
        torch.cuda.synchronize(dev)
        for k in range(3):
            phase_ms[k].append(ev[k].elapsed_time(ev[k + 1]))
        results["many"], results["sliced"], results["light"] = res_many, res_sliced, res_light
        return time.perf_counter() - t0

    for _ in range(max(args.warmup, 1)):
        one_step()
    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    times = [one_step() for _ in range(args.steps)]
    clk = clocks.stop()
    s = sum(times) / len(times)
    _, _, flags_light = results["light"]
    wrapped = int(sum(flags_light != 0)) + sum(r.flags != 0 for r in results["many"]) + \
        sum(r.flags != 0 for r in results["sliced"])
    counted = len(light) + len(results["many"]) + len(results["sliced"])
    assert counted == n_total
    line = {
        "metric": "exact model counts/s", "value": counted / s, "unit": "counts/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": s * 1000.0, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": "batch: u32 residues mod 2 primes < 2^30 (int64); heavy and sliced: u8 residues mod 8 primes <= 251 "
                 "(fp16 tensor-core dense steps)",
        "data": "synthetic",
        "config": {"workload": f"one_in_three_batch{n_total}", "counted": counted, "left_out": n_total - counted,
                   "batched_macs_le_2^24_rank_le_16": len(light), "heavy_contract_many_rank_le_26": len(many),
                   "sliced_to_rank_le_26": len(sliced),
                   "slices": sum(len(sp) for _, sp, _ in sliced),
                   "planner": "best; heavy re-planned by portfolio", "autotune": tuned, "host_threads": 1,
                   "modulus_bits": {"batch": round(sum(math.log2(q) for q in tnc.default_primes(Rc)), 1),
                                    "heavy": round(sum(math.log2(q) for q in tnc.default_primes(R8, "tc_p8")), 1)},
                   "maybe_wrapped": wrapped},
        "modular_macs_per_s": (macs_light + macs_many + macs_sliced) / s,
        "phases_ms": {"batch": statistics.mean(phase_ms[0][-args.steps:]),
                      "contract_many": statistics.mean(phase_ms[1][-args.steps:]),
                      "sliced": statistics.mean(phase_ms[2][-args.steps:])},
        "clocks": clk, "plan_s": plan_s,
    }
    print(json.dumps(line), flush=True)


def run_c5(args):
    """Learned ordering (the edge scorer of tnc.h): trained on the GPU on plan
    costs the method itself measures, then used to coarsen each network with
    the paper's best heuristic finishing it (tnc_plan_learned_opts); evaluated
    on 256 monotone 1-in-3 formulas with n = 300, m = 186 against the paper's
    heuristics (TNC_PLAN_BEST) and against the same coarsening without the
    scorer (tensor-greedy merges: what the learning adds).  Counts under
    learned and heuristic plans compared, and contraction times of both, on
    formulas small enough to contract."""
    import numpy as np
    import torch
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import tnc
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    cps = (10, 20, 30, 40, 50, 60, 70, 80)
    t0 = time.perf_counter()
    train = I.batch_one_in_three(args.train_formulas, 31337, n_lo=50, n_hi=300)
    X, T = tnc.learned_dataset_coarsen(train, states=2, cands=tnc.LEARNED_CANDIDATES, completion="bisect",
                                       max_pct=80, seed=5)
    data_s = time.perf_counter() - t0
    dp = torch.tensor(tnc.mlp_init(11), device=dev)
    pb = torch.empty(tnc.MLP_PARAMS, dtype=torch.bfloat16, device=dev)
    rng = np.random.default_rng(0)
    t0 = time.perf_counter()
    losses = []
    for rnd in range(2):
        # the second training round adds states along the learned planner's own merges
        if rnd == 1:
            t1 = time.perf_counter()
            X2, T2 = tnc.learned_dataset_coarsen(train[: len(train) // 2], states=2, cands=tnc.LEARNED_CANDIDATES,
                                                 completion="bisect", max_pct=80, seed=6, params_bf16=pb)
            data_s += time.perf_counter() - t1
            X, T = np.concatenate([X, X2]), np.concatenate([T, T2])
        perm = rng.permutation(len(T))
        losses += tnc.mlp_train(dp, torch.tensor(X[perm], device=dev), torch.tensor(T[perm], device=dev),
                                epochs=30, batch=2048, lr=2e-3 if rnd == 0 else 1e-3)
        tnc.mlp_to_bf16(dp, pb)
    train_s = time.perf_counter() - t0
    lg = lambda xs: float(np.mean(np.log2(xs)))

    def compare(evals, tag):
        t = time.perf_counter()
        best = tnc.plan_many(evals, heuristic="best", rank_cap=64)
        best_s = time.perf_counter() - t
        t = time.perf_counter()
        lp, lchose, lmacs = tnc.plan_learned_coarsen(evals, pb, completion="best", checkpoints=cps)
        l_s = time.perf_counter() - t
        gp, gchose, gmacs = tnc.plan_learned_coarsen(evals, None, completion="best", checkpoints=cps)
        bm = [p.stats.total_macs for p in best]
        return best, lp, {
            "formulas": len(evals), "workload": tag,
            "mean_log2_macs": {"best_heuristic": lg(bm), "learned_coarsen_best": lg(lmacs),
                               "greedy_coarsen_best": lg(gmacs), "kept": lg([p.stats.total_macs for p in lp])},
            "mean_max_rank": {"best_heuristic": float(np.mean([p.stats.max_rank for p in best])),
                              "kept": float(np.mean([p.stats.max_rank for p in lp]))},
            "learned_kept": int(sum(lchose)), "greedy_coarsen_kept": int(sum(gchose)),
            "learned_fewer_macs_than_best": int(sum(l < b for l, b in zip(lmacs, bm))),
            "learned_fewer_macs_than_greedy_coarsen": int(sum(l < g for l, g in zip(lmacs, gmacs))),
            "plan_s": {"best_heuristic": best_s, "learned_with_fallback": l_s}}

    n_eval = args.formulas or 256
    evals = [I.one_in_three(300, 186, 900000 + s) for s in range(n_eval)]
    _, _, big = compare(evals, "one_in_three_n300_m186")
    # contraction: formulas whose learned and heuristic plans both fit rank 28
    mid = [I.one_in_three(200, 124, 700000 + s) for s in range(48)]
    best, lp, midrep = compare(mid, "one_in_three_n200_m124")
    torch.cuda.synchronize(dev)
    both = [(f, b, l) for f, b, l in zip(mid, best, lp) if b.stats.max_rank <= 28 and l.stats.max_rank <= 28]
    agree, tl, tb = 0, 0.0, 0.0
    for f, b, l in both:
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        rl = tnc.contract(l, n_residues=20, path="tc_p8")
        torch.cuda.synchronize(dev)
        tl += time.perf_counter() - t
        t = time.perf_counter()
        rb = tnc.contract(b, n_residues=20, path="tc_p8")
        torch.cuda.synchronize(dev)
        tb += time.perf_counter() - t
        agree += int(rl.counts == rb.counts and rl.residues.tolist() == rb.residues.tolist())
    midrep["contracted"] = len(both)
    midrep["counts_identical"] = f"{agree}/{len(both)}"
    midrep["contract_s"] = {"kept_learned_or_fallback": tl, "best_heuristic": tb}
    line = {"metric": "learned ordering vs heuristic (plan MACs)",
            "value": 2 ** (big["mean_log2_macs"]["best_heuristic"] - big["mean_log2_macs"]["kept"]),
            "unit": "x fewer MACs than the best heuristic (geometric mean, kept plans)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "fp32 training, bf16 inference",
            "config": {"workload": "learned coarsening + best-heuristic completion, monotone 1-in-3",
                       "train_formulas": len(train), "train_rows": int(len(T)), "epochs": "2 rounds x 30",
                       "candidates": tnc.LEARNED_CANDIDATES, "checkpoints_pct": list(cps),
                       "label_completion": "bisect", "plan_completion": "best"},
            "train": {"dataset_s": data_s, "train_s": train_s, "loss_first": losses[0], "loss_last": losses[-1],
                      "label_variance": float(T.var())},
            "eval_n300": big, "eval_n200_contract": midrep}
    print(json.dumps(line), flush=True)


def run_fig4c(args):
    """Planner only (the exact cost before any contraction, Sec. 4): mean max
    rank of the best heuristic plan for #Cubic-Vertex-Cover on random cubic
    graphs and on random planar cubic graphs, n = 20..200 (the comparison of
    the paper's Fig. 4c; its sizes, our own generators and planners)."""
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import tnc
    seeds = args.formulas or 8
    rows = []
    t0 = time.perf_counter()
    for n in range(20, 201, 20):
        un = tnc.plan_many([I.cubic_vertex_cover(n, s) for s in range(seeds)], heuristic="best", rank_cap=64)
        pl = tnc.plan_many([I.vertex_cover_formula(n, I.random_planar_cubic_graph(n, s)) for s in range(seeds)],
                           heuristic="best", rank_cap=64)
        rows.append({"n": n, "unrestricted_mean_max_rank": statistics.mean(p.stats.max_rank for p in un),
                     "planar_mean_max_rank": statistics.mean(p.stats.max_rank for p in pl),
                     "unrestricted_mean_log2_macs": statistics.mean(math.log2(p.stats.total_macs) for p in un),
                     "planar_mean_log2_macs": statistics.mean(math.log2(p.stats.total_macs) for p in pl)})
    line = {"metric": "mean max rank vs n (planner only)", "value": rows[-1]["unrestricted_mean_max_rank"] /
            rows[-1]["planar_mean_max_rank"], "unit": "x (unrestricted / planar at n = 200)", "higher_is_better": True,
            "data": "synthetic", "config": {"workload": "cubic_vertex_cover, random vs random planar cubic graphs",
                                            "seeds_per_n": seeds, "planner": "best"},
            "plan_s": time.perf_counter() - t0, "rows": rows}
    print(json.dumps(line), flush=True)


def run_planners(args):
    """Planner only (exact plan costs before any contraction, Sec. 4), on the
    host: total MACs, output entries, max rank and planning time of the
    paper's heuristics (TNC_PLAN_BEST: tensor-greedy, tensor-METIS and
    tensor-GN, the cheapest by (max rank, MACs)) against the two-level
    planner (TNC_PLAN_COARSEN) on the formulas of the default workload (the
    first 1024), of the C4 block and of the C5 evaluation set.  The C2 and C4
    plans are capped at the ranks their runs use (32 and 30), C5's at 64."""
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import tnc
    sets = [("cubic_vertex_cover_n60_seeds0_1023", workload(0, 1024), 32),
            ("c4_cubic_vertex_cover_n180_rank_le_30", [f for _, f, _ in c4_workload()], 30),
            ("c5_one_in_three_n300_m186", [I.one_in_three(300, 186, 900000 + s) for s in range(args.formulas or 256)],
             64)]
    rows = []
    for name, forms, cap in sets:
        row = {"workload": name, "formulas": len(forms), "rank_cap": cap}
        for h in ("best", "coarsen"):
            t = time.perf_counter()
            plans = tnc.plan_many(forms, heuristic=h, rank_cap=cap)
            row[h] = {"plan_s": time.perf_counter() - t,
                      "total_macs": sum(p.stats.total_macs for p in plans),
                      "total_entries": sum(p.stats.total_entries for p in plans),
                      "mean_log2_macs": statistics.mean(math.log2(p.stats.total_macs) for p in plans),
                      "mean_max_rank": statistics.mean(p.stats.max_rank for p in plans),
                      "max_max_rank": max(p.stats.max_rank for p in plans)}
        row["macs_ratio_best_over_coarsen"] = row["best"]["total_macs"] / row["coarsen"]["total_macs"]
        rows.append(row)
    line = {"metric": "plan MACs, best heuristic / two-level planner (planner only)",
            "value": rows[0]["macs_ratio_best_over_coarsen"], "unit": "x fewer MACs (default workload)",
            "higher_is_better": True, "data": "synthetic", "host_threads": os.cpu_count(),
            "config": {"workload": "default, C4 and C5 formulas", "planners": ["best", "coarsen"]}, "rows": rows}
    print(json.dumps(line), flush=True)


def run_slicing(args):
    """Bond slicing on the rank-29 networks of C4 (#Cubic-VC, n = 180, seeds 3
    and 15): each counted whole and as 2^s slices (s = 1..4) on the
    8-bit-prime tensor-core path; reported: time, peak tensor size and
    workspace, identical counts."""
    import torch
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import slicing as S
    from paper_1805_00475_gb300 import tnc
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    R8 = 20
    stream = torch.cuda.Stream(device=dev)
    rows = []
    for seed in (3, 15):
        f = I.cubic_vertex_cover(180, seed)
        whole = tnc.plan_formula(f, heuristic="best", rank_cap=30)
        cases = [("whole", [whole], [])]
        for s in range(1, 5):
            plans_s, vs = S.sliced_plans(f, s)
            cases.append((f"s={s}", plans_s, vs))
        ref = None
        for name, plans, vs in cases:
            if name == "whole":
                nb = tnc.workspace_bytes(plans[0], R8, "tc_p8")
                run = lambda ws: tnc.contract(plans[0], n_residues=R8, path="tc_p8", workspace=ws, stream=stream)
            else:
                o, _ = tnc._opts(R8, None, "tc_p8")
                arr = (tnc.ctypes.c_void_p * len(plans))(*[p.h.value for p in plans])
                nb = int(tnc.lib().tnc_workspace_bytes_sliced(arr, len(plans), tnc.ctypes.byref(o)))
                run = lambda ws, plans=plans: tnc.contract_sliced(plans, n_residues=R8, path="tc_p8", workspace=ws,
                                                                  stream=stream)
            ws = torch.empty(nb, dtype=torch.uint8, device=dev)
            for _ in range(max(args.warmup, 1)):
                r = run(ws)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(args.steps):
                r = run(ws)
            torch.cuda.synchronize(dev)
            ms = 1000 * (time.perf_counter() - t0) / args.steps
            ref = r.counts if ref is None else ref
            assert r.counts == ref and r.flags == 0, "slices disagree with the whole network"
            rows.append({"seed": seed, "case": name, "fixed_vars": vs, "slices": len(plans),
                         "max_rank": max(p.stats.max_rank for p in plans),
                         "log2_macs": round(math.log2(sum(p.stats.total_macs for p in plans)), 2),
                         "workspace_gb": round(nb / 1e9, 2), "ms": ms})
            del ws
            torch.cuda.empty_cache()
    best = {seed: min((x for x in rows if x["seed"] == seed), key=lambda x: x["ms"]) for seed in (3, 15)}
    line = {"metric": "bond slicing on rank-29 networks", "value": sum(x["ms"] for x in rows if x["case"] == "whole") /
            sum(b["ms"] for b in best.values()), "unit": "x (whole-network time / best sliced time)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "u32 residues mod 20 primes <= 251",
            "config": {"workload": "cubic_vertex_cover_n180_seeds_3_15", "path": "tc_p8", "residues": R8},
            "cases": rows}
    print(json.dumps(line), flush=True)


def c4_block(args, dev, steps, warmup, compare):
    """16 #Cubic-VC formulas on 180 vertices: exact counts through tnc_contract
    on the 8-bit-prime tensor-core path (timed over `steps`), and, timed once
    beside it, the paths in `compare` (the 30-bit-prime limb tensor-core path
    and the CUDA-core int64 path, 8 residues each); all must give the same
    counts.  Returns the block of the bench line."""
    import torch
    from paper_1805_00475_gb300 import tnc
    Rc = 8
    t = time.perf_counter()
    kept = c4_workload(args.formulas or 16)
    plan_s = time.perf_counter() - t
    plans = [k[2] for k in kept]
    # 8-bit primes: the fewest whose product exceeds every certified bound
    bound = max(p.stats.log2_bound for p in plans)
    p8_primes, bits = [], 0.0
    for q in tnc.default_primes(53, "tc_p8"):
        if bits > bound + 1:
            break
        p8_primes.append(q)
        bits += math.log2(q)
    R8 = len(p8_primes)
    ws_bytes = max(tnc.workspace_bytes(p, R8, "tc_p8") for p in plans)
    if compare:
        ws_bytes = max(ws_bytes, max(tnc.workspace_bytes(p, Rc) for p in plans))
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    macs = sum(p.stats.total_macs for p in plans)
    dense = sum(p.stats.dense_macs for p in plans)
    dense8 = sum(p.stats.dense_macs_p8 for p in plans)
    dense_ms, device_ms, launches, io, steps_rec = [], [], [], [], []

    def one_pass(path, timed=False):
        R = R8 if path == "tc_p8" else Rc
        counts, dms, gms, nl, h2d, d2h = [], 0.0, 0.0, 0, 0, 0
        tnc.set_step_timing(timed)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for p in plans:
            r = tnc.contract(p, n_residues=R, path=path, workspace=ws, stream=stream)
            assert r.flags == 0
            counts.append(r.counts[0])
            dms += tnc.last_dense_time()[0]
            if timed:
                steps_rec.extend(tnc.last_dense_steps())
            gms += tnc.last_contract_time()
            lc = tnc.last_launch_counts()
            nl += sum(v for k, v in lc.items() if k not in ("p8_tile_n", "p8_max_chunks", "p8_swapped",
                                                            "p8_padded", "tc_split", "p8_split",
                                                            "p8_direct_out", "p8_direct_in", "p8_mn", "p8_pairs",
                                                            "p8_cta_pair"))
            nl += lc["splitk"] + lc["tc_split"] + lc["p8_split"]  # split steps launch a second kernel
            a, b = tnc.last_io_bytes()
            h2d += a
            d2h += b
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        tnc.set_step_timing(False)
        if timed:
            dense_ms.append(dms)
            device_ms.append(gms)
            launches.append(nl)
            io.append((h2d, d2h))
        return dt, counts

    for _ in range(max(warmup, 1)):
        one_pass("tc_p8")
    clocks = ClockSampler(dev.index or 0)
    clocks.start()
    time.sleep(0.3)
    times, counts = [], None
    for _ in range(steps):
        dt, counts = one_pass("tc_p8", timed=True)
        times.append(dt)
    clk = clocks.stop()
    others = {}
    for path in compare:
        others[path] = one_pass(path)
        assert others[path][1] == counts, f"the {path} path disagrees with the 8-bit-prime path"
    ttc = others["tc"][0] if "tc" in others else None
    t64 = others["int64"][0] if "int64" in others else None
    s = sum(times) / len(times)
    dms = sum(dense_ms) / len(dense_ms)
    pk, pk_kind = peaks()
    # p8 dense steps: one fp16 product (2 flops) per MAC and residue; limb
    # path: 16 limb products per MAC and residue
    p8_flops = dense8 * R8 * 2
    dev_ms = sum(device_ms) / len(device_ms)
    # per dense step: attained fraction of the peak (flops = 2 macs residues);
    # MAC-weighted by class (tile width, long or short shared dimension) and
    # the largest steps
    peak = pk["bf16_tflops"] * 1e12
    by_class = {}
    for r in steps_rec:
        key = f"tile{r['tile_n']}_{'k>=10' if r['k_log2'] >= 10 else 'k<10'}"
        c = by_class.setdefault(key, [0.0, 0.0, 0])
        c[0] += 2 * r["macs"] * r["residues"]
        c[1] += r["ms"]
        c[2] += 1
    classes = {k: {"launches": v[2] // max(1, len(dense_ms)), "share_of_dense_flops": v[0] / max(1e-30, sum(
        x[0] for x in by_class.values())), "frac": v[0] / (v[1] / 1000.0) / peak} for k, v in sorted(by_class.items())}
    top = sorted(steps_rec, key=lambda r: -r["macs"] * r["residues"])[:5]
    largest = [{"rows_log2": r["rows_log2"], "cols_log2": r["cols_log2"], "k_log2": r["k_log2"],
                "residues": r["residues"], "tile_n": r["tile_n"], "ms": r["ms"],
                "frac": 2 * r["macs"] * r["residues"] / (r["ms"] / 1000.0) / peak} for r in top]
    return {
        "workload": f"cubic_vertex_cover_n180_{len(kept)}formulas", "seeds": [k[0] for k in kept],
        "max_ranks": [p.stats.max_rank for p in plans], "planner": "best",
        "value": len(plans) / s, "unit": "counts/s", "ms_per_step": s * 1000.0, "steps": steps, "warmup": warmup,
        "step": "tnc_contract of every formula, one after another, host result buffers (e2e through the C ABI: "
                "descriptor uploads and result reads inside)",
        "path": "tc_p8", "residues": R8, "primes": p8_primes, "log2_bound_max": round(bound, 2),
        "dtype": "u8 residues mod primes <= 251; dense steps fp16 (exact), fp32 accumulate reduced every 1024",
        "modular_macs_per_s": macs * R8 / s,
        "device_ms_per_step": dev_ms, "gpu_launches_per_step": sum(launches) / len(launches),
        "e2e": {"value": len(plans) / s, "unit": "counts/s", "h2d_bytes_per_step": io[-1][0],
                "d2h_bytes_per_step": io[-1][1],
                "note": "the timed step is already end to end: tnc_contract uploads each plan's descriptors "
                        "and returns host counts"},
        "tc_limb_path": None if ttc is None else {
            "residues": Rc, "ms_per_step": ttc * 1000.0, "speedup_tc_p8": ttc / s,
            "limb_tflops": dense * Rc * 16 * 2 / ttc / 1e12},
        "int64_path": None if t64 is None else {
            "residues": Rc, "ms_per_step": t64 * 1000.0, "modular_macs_per_s": macs * Rc / t64,
            "speedup_tc_p8": t64 / s, "speedup_tc_limb": t64 / ttc if ttc else None},
        "counts_identical_across_paths": ["tc_p8"] + list(others),
        "roofline": {"bound": "tensor", "achieved": p8_flops / dms / 1e9, "peak": pk["bf16_tflops"],
                     "unit": "TFLOP/s", "frac": p8_flops / dms / 1e9 / pk["bf16_tflops"], "traffic": None,
                     "peak_source": f"{pk_kind} bf16 dense burst (MEASURED_PEAKS.json); fp16 has the same dense rate",
                     "kernel": "dense steps: p8_pack + p8_gemm_kernel (+ split sum), CUDA events around each",
                     "dense_ms_per_step": dms, "dense_share_of_device_time": dms / dev_ms,
                     "whole_contraction_tflops": p8_flops / s / 1e12,
                     "algorithmic_flops_per_step": p8_flops,
                     "flops": "sum over dense steps of 2^(a+b-k) x residues x 2",
                     "per_step": {"by_class": classes, "largest_launches": largest,
                                  "note": "fraction of the measured peak per dense launch (packing + GEMM), from "
                                          "CUDA events around each launch"}},
        "clocks": clk, "plan_s": plan_s,
        "counts_log2": [round(math.log2(c), 2) for c in counts],
    }


def c4_cpu_baseline(dev, budget_s=30.0):
    """The oracle cannot contract the rank-29 C4 networks (tensors of 2^29 big
    integers); it is timed instead on the largest #Cubic-VC formula it finishes
    in seconds (n = 100, seed 11, tensor-greedy, rank 24), next to the
    8-bit-prime path on the same formula."""
    import oracle
    import torch
    from paper_1805_00475_gb300 import instances as I
    from paper_1805_00475_gb300 import tnc
    f = I.cubic_vertex_cover(100, 11)
    oracle.build()
    t = time.perf_counter()
    exact = oracle.count(f, max_rank=26)
    cpu_s = time.perf_counter() - t
    p = tnc.plan_formula(f, heuristic="greedy", rank_cap=26)
    R8 = 0
    bits = 0.0
    for q in tnc.default_primes(53, "tc_p8"):
        if bits > p.stats.log2_bound + 1:
            break
        bits += math.log2(q)
        R8 += 1
    r = tnc.contract(p, n_residues=R8, path="tc_p8")
    assert r.counts == exact
    torch.cuda.synchronize(dev)
    t = time.perf_counter()
    for _ in range(5):
        tnc.contract(p, n_residues=R8, path="tc_p8")
    torch.cuda.synchronize(dev)
    gpu_s = (time.perf_counter() - t) / 5
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": 1.0 / cpu_s, "unit": "counts/s", "cores": threads, "kind": "oracle",
            "sample": f"#Cubic-VC n=100 seed 11 (tensor-greedy, rank 24; C4's rank-29 networks are beyond the "
                      f"oracle): oracle {cpu_s:.1f} s, tc_p8 path {gpu_s * 1000:.1f} ms on the same formula, "
                      f"same count"}


def run_c4(args):
    """The C4 comparison alone (bench.py --config c4)."""
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    blk = c4_block(args, dev, args.steps, args.warmup, [x for x in args.c4_compare.split(",") if x])
    line = {"metric": METRIC, "value": blk["value"], "unit": "counts/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": blk["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": blk["dtype"], "data": "synthetic",
            "config": {"workload": blk["workload"], "seeds": blk["seeds"], "max_ranks": blk["max_ranks"],
                       "planner": "best", "path": "tc_p8", "residues": blk["residues"], "primes": blk["primes"],
                       "l2": "inputs (up to 18 GB of tensors) far above L2"},
            "modular_macs_per_s": blk["modular_macs_per_s"], "tc_limb_path": blk["tc_limb_path"],
            "int64_path": blk["int64_path"], "roofline": blk["roofline"], "clocks": blk["clocks"],
            "plan_s": blk["plan_s"], "counts_log2": blk["counts_log2"],
            "gpu_launches": int(blk["gpu_launches_per_step"] * args.steps),
            "e2e": blk["e2e"],
            "cpu_baseline": c4_cpu_baseline(dev)}
    print(json.dumps(line), flush=True)


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of
# the C2 batch kernel come from an ncu capture summarised in this profile; the
# figure is used only while the kernel's device sources are the ones captured
# (their SHA-256 is recorded beside it), else the line reports null.
C2_PROFILE = os.path.join(ROOT, "profiles", "batch_kernel_cubic_vc_n60_R4.md")
C2_KERNEL_SOURCES = ["paper_1805_00475_gb300/csrc/kernels.cuh", "paper_1805_00475_gb300/csrc/modarith.cuh",
                     "paper_1805_00475_gb300/csrc/step_desc.h"]


def kernel_source_sha(paths) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def captured_traffic(profile: str, sources, planner: str, plan_macs: float = None) -> tuple:
    """(bytes per launch, note) from the profile's 'traffic_bytes_per_launch
    = B, kernel_source_sha = H, planner = P[, plan_macs = M]' line if H
    matches the current sources, P the planner of this run and M (the
    algorithmic MACs of the captured launch) this launch's (the plans fix the
    launch's work), else (None, why)."""
    import re
    try:
        with open(profile) as fh:
            txt = fh.read()
    except OSError:
        return None, "no profile"
    m = re.search(r"traffic_bytes_per_launch\s*=\s*([0-9.eE+]+)\s*,\s*kernel_source_sha\s*=\s*([0-9a-f]+)"
                  r"\s*,\s*planner\s*=\s*(\w+)(?:\s*,\s*plan_macs\s*=\s*([0-9]+))?", txt)
    if not m:
        return None, "no traffic line in the profile"
    sha = kernel_source_sha(sources)
    if m.group(2) != sha:
        return None, f"kernel changed since the capture (sources {sha}, captured {m.group(2)})"
    if m.group(3) != planner:
        return None, f"captured with planner {m.group(3)}, this run plans with {planner}"
    if m.group(4) is not None and plan_macs is not None and int(m.group(4)) != int(round(plan_macs)):
        return None, f"plans changed since the capture ({int(round(plan_macs))} MACs per launch, captured {m.group(4)})"
    return float(m.group(1)), f"ncu capture of this workload and kernel ({os.path.relpath(profile, ROOT)})"


def run_tnc(args):
    import torch
    import torch.distributed as dist
    from paper_1805_00475_gb300 import tnc

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group(backend="nccl", init_method="env://", device_id=dev)

    forms = workload(rank, args.batch)
    t = time.perf_counter()
    plans = tnc.plan_many(forms, heuristic=args.planner)
    plan_s = time.perf_counter() - t
    macs = sum(p.stats.total_macs for p in plans) * R
    entries = sum(p.stats.total_entries for p in plans)
    alg_bytes = entries * 4 * R
    batch = tnc.Batch(plans, n_residues=R)
    h2d, d2h, n_entries, kpl = batch.info()
    ws = torch.empty(batch.workspace_bytes(), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)
    batch.upload(ws, stream)
    t = time.perf_counter()
    if args.launch:
        shape = [int(x) for x in args.launch.split(",")] + [0]
        tuned_threads, tuned_smem, tuned_ctas = shape[:3]
        batch.set_launch(tuned_threads, tuned_smem, tuned_ctas)
    else:
        tuned_threads, tuned_smem, tuned_ctas = batch.autotune(ws, stream)
    tune_s = time.perf_counter() - t
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            flush.fill_(1)
            batch.launch(ws, stream)
    stream.synchronize()
    # correctness of what is timed: spot-check a few formulas against exact counts
    # computed once above the timed region by the CPU oracle is done in the tests;
    # here the device status and a residue sanity check suffice
    out = batch.download(ws, stream)
    assert all(o.flags == 0 for o in out), "uncertified CRT in the workload"

    # Blocks of exactly K timed steps, each bracketed by a barrier and a
    # synchronize, repeated until the timed steps cover --min-timed-s of
    # device time (so that the clock record spans the measurement); every
    # rank runs the same number of blocks (the count is agreed on first).
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]

    def timed_block():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        with torch.cuda.stream(stream):
            for s in range(args.steps):
                flush.fill_(s & 0xFF)
                starts[s].record(stream)
                batch.launch(ws, stream)
                ends[s].record(stream)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        return sum(a.elapsed_time(b) for a, b in zip(starts, ends))

    probe_ms = timed_block()
    n_blocks = max(1, min(400, int(math.ceil(args.min_timed_s * 1000.0 / max(probe_ms, 1e-3)))))
    if world > 1:
        n_blocks = int(max_over_ranks(float(n_blocks), dist, dev))
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    wall0 = time.perf_counter()
    block_ms = [timed_block() for _ in range(n_blocks)]
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    total_ms = sum(block_ms)
    if world > 1:
        total_ms = max_over_ranks(total_ms, dist, dev)
    ms = total_ms / (args.steps * n_blocks)
    value = args.batch * world / (ms / 1000.0)

    # end to end through the C ABI with host buffers: every step uploads the
    # packed formulas from pinned host memory, launches, and reads the exact
    # counts back into host buffers (tnc_batch_upload / _launch /
    # _download_flat).  The formulas are split into a few batches, each with
    # its workspace and stream and the timed launch shape: upload and launch
    # are asynchronous, so a batch's upload overlaps the previous batch's
    # kernel; the downloads then wait for each stream.
    e2e = None
    if not args.no_e2e:
        e2e_steps = max(3, min(args.steps, 10))
        shares = [float(x) for x in args.e2e_split.split(",") if x]
        acc, cuts = 0.0, [0]
        for x in shares:
            acc += x
            cuts.append(min(len(plans), int(round(len(plans) * acc / sum(shares)))))
        cuts = sorted(set(cuts))
        nch = len(cuts) - 1
        chunks = []
        for c in range(nch):
            b = tnc.Batch(plans[cuts[c]:cuts[c + 1]], n_residues=R)
            b.set_launch(tuned_threads, tuned_smem, tuned_ctas)
            chunks.append((b, torch.empty(b.workspace_bytes(), dtype=torch.uint8, device=dev),
                           torch.cuda.Stream(device=dev)))
        h2d_e = sum(b.info()[0] for b, _, _ in chunks)
        d2h_e = sum(b.info()[1] for b, _, _ in chunks)

        def e2e_step(hosts):
            for b, w, st in chunks:
                b.upload(w, st)
                b.launch(w, st)
            return [b.download_flat(w, st, h) for (b, w, st), h in zip(chunks, hosts)]

        hosts = [None] * nch
        for _ in range(2):
            hosts = e2e_step(hosts)
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        for _ in range(e2e_steps):
            hosts = e2e_step(hosts)
        e2e_s = (time.perf_counter() - t) / e2e_steps
        assert sum(h[0].shape[0] for h in hosts) == args.batch and not any(h[2].any() for h in hosts)
        e2e = {"value": args.batch * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d_e),
               "d2h_bytes_per_step": int(d2h_e), "ms_per_step": e2e_s * 1000.0, "batches": nch,
               "includes": "packed-formula H2D (pinned) + persistent launches + residue and CRT-limb D2H "
                           "into host arrays per step, the formulas in batches on their own streams; "
                           "planning and packing excluded"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    pk, pk_kind = peaks()
    achieved_gbs = alg_bytes / (ms / 1000.0) / 1e9
    achieved_macs = macs / (ms / 1000.0)
    probe = tnc.probe_modmac(8192, stream=stream)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    # integer-pipe ceiling from unit counts and clocks: per SM 4 partitions x 16
    # lanes issue a 32-bit IMAD per clock; a residue MAC (u32 x u32 + u64) is one
    # 64-bit-result IMAD, two issue slots; clock = max SM clock
    alu_peak = sms * 4 * 16 / 2 * pk.get("sm_max_mhz", 2070.0) * 1e6
    default_shape = args.batch == 8192 and not args.launch
    traffic, traffic_src = captured_traffic(C2_PROFILE, C2_KERNEL_SOURCES, args.planner, macs) if default_shape else \
        (None, "captured for the default workload only")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32 residues, int64 accumulate", "data": "synthetic",
        "config": config(args, world),
        "modular_macs_per_s": macs * world / (ms / 1000.0),
        "roofline": {"bound": "alu", "achieved": achieved_macs / 1e12, "peak": probe / 1e12,
                     "unit": "Tmodmac/s", "frac": achieved_macs / probe,
                     "traffic": traffic, "traffic_source": traffic_src,
                     "peak_source": "measured in this run: tnc_probe_modmac (4 residues per thread, u32 x u32 "
                                    "products in 64-bit sums reduced every 16th product, operands in registers, "
                                    "all SMs)",
                     "derived_peak": alu_peak / 1e12, "frac_of_derived": achieved_macs / alu_peak,
                     "derived_peak_source": "SMs x 64 IMAD lanes / 2 slots per 64-bit MAC x max SM clock",
                     "kernel": "batch_kernel<4>", "algorithmic_macs_per_launch": macs,
                     "algorithmic_bytes_per_launch": alg_bytes, "bytes_per_s_vs_hbm": achieved_gbs / pk["hbm_gbs"]},
        "autotune": {"threads": tuned_threads, "smem_arena_bytes": tuned_smem, "ctas_per_sm_cap": tuned_ctas,
                     "seconds": tune_s},
        "clocks": clk,
        "gpu_launches": kpl * args.steps * n_blocks,
        "timing": {"blocks": n_blocks, "steps_per_block": args.steps, "timed_steps": n_blocks * args.steps,
                   "device_ms_timed": sum(block_ms),
                   "how": "blocks of K steps, each between barrier + synchronize, CUDA events per step on the "
                          "launching stream, L2 flushed before every step; ms_per_step = all timed steps' mean"},
        "plan_s": plan_s,
        "wall_s_timed_region": wall,
    }
    if e2e:
        line["e2e"] = e2e
    # the oracle on the host cores, on a bounded sample of the same workload
    done, el, threads = oracle_sample(forms, args.cpu_seconds)
    line["cpu_baseline"] = {"value": done / el, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": f"first {done} formulas of the workload ({el:.1f} s, C bigint oracle)"}
    if not args.no_c4 and world == 1:
        del ws, flush
        torch.cuda.empty_cache()
        blk = c4_block(args, dev, max(3, min(args.steps, 10)), 2, ["tc", "int64"])
        blk["cpu_baseline"] = c4_cpu_baseline(dev)
        line["c4"] = blk
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "c4":
        run_c4(args)
    elif args.config == "slicing":
        run_slicing(args)
    elif args.config == "planners":
        run_planners(args)
    elif args.config == "fig4c":
        run_fig4c(args)
    elif args.config == "c3":
        run_c3(args)
    elif args.config == "c5":
        run_c5(args)
    else:
        run_tnc(args)


if __name__ == "__main__":
    main()
