"""Thin Python binding of libtnc (include/tnc.h): argument marshalling only.

Every step of the counting path -- leaf tensors, pairwise contractions, residue
extraction, CRT -- runs in libtnc's CUDA kernels; planning runs in libtnc's C++
host code.  PyTorch is used for device memory (the workspace) and streams only.
The binding raises if the library is missing: there is no fallback path.

Names follow the C ABI: build_network, plan, workspace_bytes, contract,
Batch.{create, upload, launch, download}, contract_batch.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libtnc.so")

TNC_OK = 0
ERRORS = {-1: "TNC_ERR_INVALID", -2: "TNC_ERR_TOO_LARGE", -3: "TNC_ERR_CUDA", -4: "TNC_ERR_BUFFER",
          -5: "TNC_ERR_TIMEOUT", -6: "TNC_ERR_NOMEM"}
HEURISTICS = {"greedy": 0, "bisect": 1, "gn": 2, "explicit": 3, "best": 4, "portfolio": 5, "coarsen": 6}
PATHS = {"int64": 0, "tc": 1, "tc_p8": 2}
TNC_MAYBE_WRAPPED = 1
INJECT = {"none": 0, "nomem": 1, "plan": 2, "launch": 3, "timeout": 4}

# every symbol include/tnc.h declares
EXPORTS = [
    "tnc_version", "tnc_last_error", "tnc_default_primes", "tnc_default_primes_p8", "tnc_build_network", "tnc_network_info",
    "tnc_free_network", "tnc_plan", "tnc_plan_many", "tnc_plan_sliced", "tnc_slice_network", "tnc_network_formula", "tnc_plan_steps", "tnc_free_plan", "tnc_workspace_bytes", "tnc_workspace_bytes_opts", "tnc_set_step_timing", "tnc_last_dense_time", "tnc_last_contract_time", "tnc_last_launch_counts", "tnc_last_io_bytes", "tnc_last_dense_steps", "tnc_workspace_bytes_sliced", "tnc_contract_sliced",
    "tnc_workspace_bytes_many", "tnc_contract_many",
    "tnc_contract", "tnc_crt_host", "tnc_residue_add_host", "tnc_batch_create", "tnc_batch_workspace_bytes", "tnc_batch_info", "tnc_batch_upload", "tnc_batch_autotune", "tnc_batch_set_launch", "tnc_batch_get_launch",
    "tnc_batch_launch", "tnc_batch_download", "tnc_batch_download_flat", "tnc_batch_status", "tnc_free_batch",
    "tnc_contract_batch", "tnc_contract_noalloc", "tnc_probe_modmac", "tnc_inject_failure", "tnc_learned_save",
    "tnc_learned_load",
    "tnc_mlp_init", "tnc_learned_dataset", "tnc_learned_dataset_on_policy", "tnc_mlp_forward", "tnc_mlp_backward_scratch_floats",
    "tnc_mlp_backward", "tnc_mlp_adam", "tnc_mlp_train_workspace_bytes", "tnc_mlp_train", "tnc_mlp_to_bf16",
    "tnc_mlp_forward_bf16", "tnc_plan_learned_workspace_bytes", "tnc_plan_learned_many", "tnc_plan_learned_opts",
    "tnc_learned_dataset_opts",
]
MLP_FEATURES = 16
MLP_HIDDEN = 128
MLP_PARAMS = MLP_FEATURES * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1
LEARNED_CANDIDATES = 8
NOALLOC_SCRATCH_BYTES = 32 << 20


class TncError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class _Formula(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int32), ("n_cons", ctypes.c_int32),
                ("arity", ctypes.POINTER(ctypes.c_int32)), ("var_of", ctypes.POINTER(ctypes.c_int32)),
                ("kind", ctypes.POINTER(ctypes.c_uint8)), ("table", ctypes.POINTER(ctypes.c_uint32)),
                ("n_open", ctypes.c_int32), ("open_vars", ctypes.POINTER(ctypes.c_int32))]


class _PlanOpts(ctypes.Structure):
    _fields_ = [("heuristic", ctypes.c_int32), ("rank_cap", ctypes.c_int32), ("tries", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("order", ctypes.POINTER(ctypes.c_int32)),
                ("n_order", ctypes.c_int32)]


class _PlanStats(ctypes.Structure):
    _fields_ = [("max_rank", ctypes.c_int32), ("n_steps", ctypes.c_int32), ("n_leaves", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("total_macs", ctypes.c_double),
                ("total_entries", ctypes.c_double), ("log2_bound", ctypes.c_double),
                ("arena_entries", ctypes.c_uint64), ("batch_arena_entries", ctypes.c_uint64),
                ("n_dense_steps", ctypes.c_int32), ("dense_macs", ctypes.c_double),
                ("n_dense_steps_p8", ctypes.c_int32), ("dense_macs_p8", ctypes.c_double),
                ("n_direct_p8", ctypes.c_int32), ("p8_arena_entries", ctypes.c_uint64)]


class _LaunchCounts(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("leaf_fill", "level", "grid_step", "splitk", "tc_gemm", "tc_split",
                                              "p8_pack", "p8_gemm", "p8_split")] + \
               [("p8_tile_n", ctypes.c_int32 * 5)] + \
               [(n, ctypes.c_int32) for n in ("p8_max_chunks", "p8_swapped", "p8_padded", "extract", "crt",
                                              "p8_direct_out", "p8_direct_in", "p8_mn", "p8_pairs", "outer",
                                              "p8_cta_pair")]


class _LearnedOpts(ctypes.Structure):
    _fields_ = [("states", ctypes.c_int32), ("cands", ctypes.c_int32), ("completion", ctypes.c_int32),
                ("n_checkpoints", ctypes.c_int32), ("checkpoints", ctypes.c_int32 * 8), ("max_pct", ctypes.c_int32),
                ("seed", ctypes.c_uint64)]


class _DenseStepTime(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double), ("macs", ctypes.c_double)] + \
               [(n, ctypes.c_int32) for n in ("rows_log2", "cols_log2", "k_log2", "residues", "tile_n", "log_split")]


class _ContractOpts(ctypes.Structure):
    _fields_ = [("path", ctypes.c_int32), ("n_residues", ctypes.c_int32),
                ("primes", ctypes.POINTER(ctypes.c_uint32))]


class _Count(ctypes.Structure):
    _fields_ = [("residues", ctypes.POINTER(ctypes.c_uint32)), ("limbs", ctypes.POINTER(ctypes.c_uint32)),
                ("cap_out", ctypes.c_int32), ("cap_limbs", ctypes.c_int32), ("n_out", ctypes.c_int32),
                ("n_limbs", ctypes.c_int32), ("flags", ctypes.c_uint32)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return LIB_PATH


def lib():
    """Load libtnc.so (built by paper_1805_00475_gb300.build); raise if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtnc.so not built ({LIB_PATH}); run python -m paper_1805_00475_gb300.build")
        L = ctypes.CDLL(LIB_PATH)
        vp, sz = ctypes.c_void_p, ctypes.c_size_t
        i32, u32p, i32p = ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_int32)
        sig = {
            "tnc_version": ([], ctypes.c_char_p),
            "tnc_last_error": ([], ctypes.c_char_p),
            "tnc_default_primes": ([i32, u32p], ctypes.c_int),
            "tnc_default_primes_p8": ([i32, u32p], ctypes.c_int),
            "tnc_build_network": ([ctypes.POINTER(_Formula), ctypes.POINTER(vp)], ctypes.c_int),
            "tnc_network_info": ([vp, i32p, i32p, i32p], ctypes.c_int),
            "tnc_free_network": ([vp], None),
            "tnc_plan": ([vp, ctypes.POINTER(_PlanOpts), ctypes.POINTER(vp), ctypes.POINTER(_PlanStats)],
                         ctypes.c_int),
            "tnc_plan_many": ([ctypes.POINTER(vp), i32, ctypes.POINTER(_PlanOpts), ctypes.POINTER(vp),
                               ctypes.POINTER(_PlanStats)], ctypes.c_int),
            "tnc_plan_steps": ([vp, i32p, i32p, i32], ctypes.c_int),
            "tnc_plan_sliced": ([vp, i32, ctypes.POINTER(_PlanOpts), ctypes.POINTER(vp), i32p,
                                 ctypes.POINTER(_PlanStats)], ctypes.c_int),
            "tnc_slice_network": ([vp, i32, i32p, ctypes.c_uint32, ctypes.POINTER(vp)], ctypes.c_int),
            "tnc_network_formula": ([vp, i32p, i32p, i32p, i32p, i32p, i32p, i32p, ctypes.POINTER(ctypes.c_uint8),
                                     u32p, i32p], ctypes.c_int),
            "tnc_free_plan": ([vp], None),
            "tnc_workspace_bytes": ([vp, i32], sz),
            "tnc_workspace_bytes_opts": ([vp, vp], sz),
            "tnc_set_step_timing": ([i32], None),
            "tnc_last_dense_time": ([ctypes.POINTER(ctypes.c_double), i32p], ctypes.c_int),
            "tnc_last_contract_time": ([ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "tnc_last_launch_counts": ([ctypes.POINTER(_LaunchCounts)], ctypes.c_int),
            "tnc_last_io_bytes": ([ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)], ctypes.c_int),
            "tnc_last_dense_steps": ([ctypes.POINTER(_DenseStepTime), i32, i32p], ctypes.c_int),
            "tnc_workspace_bytes_sliced": ([vp, i32, vp], sz),
            "tnc_contract_sliced": ([vp, i32, vp, vp, sz, vp, vp], ctypes.c_int),
            "tnc_workspace_bytes_many": ([vp, i32, vp, i32], sz),
            "tnc_contract_many": ([vp, i32, vp, vp, sz, vp, vp], ctypes.c_int),
            "tnc_contract": ([vp, ctypes.POINTER(_ContractOpts), vp, sz, vp, ctypes.POINTER(_Count)],
                             ctypes.c_int),
            "tnc_batch_create": ([ctypes.POINTER(vp), i32, ctypes.POINTER(_ContractOpts), ctypes.POINTER(vp)],
                                 ctypes.c_int),
            "tnc_crt_host": ([u32p, i32, u32p, ctypes.c_int64, u32p, i32, i32p], ctypes.c_int),
            "tnc_residue_add_host": ([u32p, i32, u32p, u32p, ctypes.c_int64], ctypes.c_int),
            "tnc_batch_workspace_bytes": ([vp], sz),
            "tnc_batch_info": ([vp, ctypes.POINTER(sz), ctypes.POINTER(sz), ctypes.POINTER(ctypes.c_uint64),
                                i32p], ctypes.c_int),
            "tnc_batch_upload": ([vp, vp, sz, vp], ctypes.c_int),
            "tnc_batch_launch": ([vp, vp, vp], ctypes.c_int),
            "tnc_batch_autotune": ([vp, vp, vp, i32p, i32p, i32p], ctypes.c_int),
            "tnc_batch_set_launch": ([vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32], ctypes.c_int),
            "tnc_batch_get_launch": ([vp, i32p, i32p, i32p], ctypes.c_int),
            "tnc_inject_failure": ([i32, i32], ctypes.c_int),
            "tnc_learned_save": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "tnc_learned_load": ([ctypes.c_char_p, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "tnc_batch_download": ([vp, vp, vp, ctypes.POINTER(_Count)], ctypes.c_int),
            "tnc_batch_download_flat": ([vp, vp, vp, u32p, u32p, u32p], ctypes.c_int),
            "tnc_batch_status": ([vp, vp, vp], ctypes.c_int),
            "tnc_free_batch": ([vp], None),
            "tnc_contract_batch": ([ctypes.POINTER(vp), i32, ctypes.POINTER(_ContractOpts), vp, sz, vp,
                                    ctypes.POINTER(_Count)], ctypes.c_int),
            "tnc_probe_modmac": ([vp, i32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "tnc_mlp_init": ([ctypes.c_uint64, ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "tnc_learned_dataset": ([ctypes.POINTER(vp), i32, i32, i32, ctypes.c_uint64,
                                     ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                     ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
            "tnc_learned_dataset_on_policy": ([ctypes.POINTER(vp), i32, vp, vp, sz, vp, i32, ctypes.c_uint64,
                                               ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                               ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
            "tnc_mlp_forward": ([vp, vp, ctypes.c_int64, vp, vp, vp, vp], ctypes.c_int),
            "tnc_mlp_backward_scratch_floats": ([ctypes.c_int64], sz),
            "tnc_mlp_backward": ([vp, vp, vp, vp, vp, vp, ctypes.c_int64, vp, vp, vp], ctypes.c_int),
            "tnc_mlp_adam": ([vp, vp, vp, vp, i32, ctypes.c_float, vp], ctypes.c_int),
            "tnc_mlp_train_workspace_bytes": ([i32], sz),
            "tnc_mlp_train": ([vp, vp, vp, ctypes.c_int64, i32, i32, ctypes.c_float, vp, sz, vp,
                               ctypes.POINTER(ctypes.c_float)], ctypes.c_int),
            "tnc_mlp_to_bf16": ([vp, vp, vp], ctypes.c_int),
            "tnc_mlp_forward_bf16": ([vp, vp, ctypes.c_int64, vp, vp], ctypes.c_int),
            "tnc_plan_learned_workspace_bytes": ([i32], sz),
            "tnc_plan_learned_many": ([ctypes.POINTER(vp), i32, vp, ctypes.POINTER(_PlanOpts), vp, sz, vp,
                                       ctypes.POINTER(vp), ctypes.POINTER(_PlanStats), i32p,
                                       ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "tnc_contract_noalloc": ([vp, ctypes.POINTER(_ContractOpts), vp, ctypes.POINTER(_Count)], ctypes.c_int),
            "tnc_plan_learned_opts": ([ctypes.POINTER(vp), i32, vp, ctypes.POINTER(_LearnedOpts),
                                       ctypes.POINTER(_PlanOpts), vp, sz, vp, ctypes.POINTER(vp),
                                       ctypes.POINTER(_PlanStats), i32p, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
            "tnc_learned_dataset_opts": ([ctypes.POINTER(vp), i32, ctypes.POINTER(_LearnedOpts), vp, vp, sz, vp,
                                          ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                          ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
        return L


def _check(rc: int):
    if rc != TNC_OK:
        raise TncError(rc, lib().tnc_last_error().decode())


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def version() -> str:
    return lib().tnc_version().decode()


def default_primes(n: int, path: str = "int64") -> List[int]:
    """The path's default primes (tnc_default_primes; tnc_default_primes_p8 for "tc_p8")."""
    out = np.zeros(max(n, 1), dtype=np.uint32)
    fn = lib().tnc_default_primes_p8 if path == "tc_p8" else lib().tnc_default_primes
    _check(fn(n, _p(out, ctypes.c_uint32)))
    return [int(x) for x in out[:n]]


# ------------------------------------------------------------------ network

class Network:
    """tnc_network_t: the COPY + clause tensor network of a formula (Sec. 2.1)."""

    def __init__(self, handle):
        self.h = handle

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tnc_free_network(self.h)
            self.h = None

    def info(self) -> Tuple[int, int, int]:
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tnc_network_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value


def build_network(formula) -> Network:
    """formula: any object with n_vars, clauses, kinds, tables, open_vars."""
    arity = np.array([len(c) for c in formula.clauses] or [0], dtype=np.int32)
    var_of = np.array([v for c in formula.clauses for v in c] or [0], dtype=np.int32)
    kind = np.array(list(formula.kinds) or [0], dtype=np.uint8)
    tab = []
    for k, t in zip(formula.kinds, getattr(formula, "tables", None) or [None] * len(formula.kinds)):
        if k == 3:
            tab.extend(int(x) for x in t)
    table = np.array(tab or [0], dtype=np.uint32)
    opens = np.array(list(formula.open_vars) or [0], dtype=np.int32)
    f = _Formula(formula.n_vars, len(formula.clauses), _p(arity, ctypes.c_int32), _p(var_of, ctypes.c_int32),
                 _p(kind, ctypes.c_uint8), _p(table, ctypes.c_uint32), len(formula.open_vars),
                 _p(opens, ctypes.c_int32))
    h = ctypes.c_void_p()
    _check(lib().tnc_build_network(ctypes.byref(f), ctypes.byref(h)))
    return Network(h)


# ------------------------------------------------------------------ plan

@dataclass
class PlanStats:
    max_rank: int
    n_steps: int
    n_leaves: int
    depth: int
    total_macs: float
    total_entries: float
    log2_bound: float
    arena_entries: int = 0
    batch_arena_entries: int = 0
    n_dense_steps: int = 0
    dense_macs: float = 0.0
    n_dense_steps_p8: int = 0
    dense_macs_p8: float = 0.0
    n_direct_p8: int = 0
    p8_arena_entries: int = 0


class Plan:
    """tnc_plan_t: contraction tree + lowered descriptors."""

    def __init__(self, handle, stats: PlanStats, n_open: int):
        self.h = handle
        self.stats = stats
        self.n_open = n_open

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tnc_free_plan(self.h)
            self.h = None

    def steps(self) -> List[Tuple[int, int]]:
        n = self.stats.n_steps
        l = np.zeros(max(n, 1), dtype=np.int32)
        r = np.zeros(max(n, 1), dtype=np.int32)
        _check(lib().tnc_plan_steps(self.h, _p(l, ctypes.c_int32), _p(r, ctypes.c_int32), n))
        return [(int(a), int(b)) for a, b in zip(l[:n], r[:n])]


def plan(network: Network, heuristic: str = "bisect", rank_cap: int = 32, tries: int = 2, seed: int = 0,
         order: Optional[Sequence[Tuple[int, int]]] = None, n_open: int = 0) -> Plan:
    ordr = np.array([x for p in (order or []) for x in p] or [0], dtype=np.int32)
    o = _PlanOpts(HEURISTICS[heuristic] if order is None else HEURISTICS["explicit"], rank_cap, tries, seed,
                  _p(ordr, ctypes.c_int32), len(order or []))
    st = _PlanStats()
    h = ctypes.c_void_p()
    _check(lib().tnc_plan(network.h, ctypes.byref(o), ctypes.byref(h), ctypes.byref(st)))
    return Plan(h, _stats(st), n_open)


def _stats(st: _PlanStats) -> PlanStats:
    return PlanStats(st.max_rank, st.n_steps, st.n_leaves, st.depth, st.total_macs, st.total_entries,
                     st.log2_bound, int(st.arena_entries), int(st.batch_arena_entries), int(st.n_dense_steps),
                     float(st.dense_macs), int(st.n_dense_steps_p8), float(st.dense_macs_p8),
                     int(st.n_direct_p8), int(st.p8_arena_entries))


def plan_many(formulas, heuristic: str = "bisect", rank_cap: int = 32, tries: int = 2, seed: int = 0
              ) -> List[Plan]:
    """Build and plan many formulas; planning runs in parallel on the host
    cores inside libtnc (tnc_plan_many)."""
    nets = [build_network(f) for f in formulas]
    n = len(nets)
    arr = (ctypes.c_void_p * n)(*[x.h.value for x in nets])
    outs = (ctypes.c_void_p * n)()
    sts = (_PlanStats * n)()
    ordr = np.zeros(1, dtype=np.int32)
    o = _PlanOpts(HEURISTICS[heuristic], rank_cap, tries, seed, _p(ordr, ctypes.c_int32), 0)
    _check(lib().tnc_plan_many(arr, n, ctypes.byref(o), outs, sts))
    return [Plan(ctypes.c_void_p(outs[i]), _stats(sts[i]), len(formulas[i].open_vars)) for i in range(n)]


def plan_sliced(formula, s: int, heuristic: str = "best", rank_cap: int = 64, tries: int = 2, seed: int = 0
                ) -> Tuple[List[Plan], List[int]]:
    """tnc_plan_sliced: the s variables the library chooses and the plans of
    the 2^s slices (slice j fixes vars[i] = bit i of j)."""
    net = build_network(formula)
    n = 1 << s
    outs = (ctypes.c_void_p * n)()
    sts = (_PlanStats * n)()
    vs = np.zeros(max(s, 1), dtype=np.int32)
    ordr = np.zeros(1, dtype=np.int32)
    o = _PlanOpts(HEURISTICS[heuristic], rank_cap, tries, seed, _p(ordr, ctypes.c_int32), 0)
    _check(lib().tnc_plan_sliced(net.h, s, ctypes.byref(o), outs, _p(vs, ctypes.c_int32), sts))
    n_open = len(formula.open_vars)
    return [Plan(ctypes.c_void_p(outs[i]), _stats(sts[i]), n_open) for i in range(n)], [int(v) for v in vs[:s]]


class FormulaView:
    """A formula read back from a network (tnc_network_formula): the
    attributes the oracle and the instance generators use."""

    def __init__(self, n_vars, clauses, kinds, tables, open_vars):
        self.n_vars, self.clauses, self.kinds, self.tables, self.open_vars = n_vars, clauses, kinds, tables, open_vars
        self.n_cons = len(clauses)
        self.name = "network"


def network_formula(net: Network) -> FormulaView:
    a = [ctypes.c_int32() for _ in range(5)]
    _check(lib().tnc_network_formula(net.h, *[ctypes.byref(x) for x in a], None, None, None, None, None))
    nv, nc, nocc, ntab, nopen = [x.value for x in a]
    arity = np.zeros(max(nc, 1), dtype=np.int32)
    var_of = np.zeros(max(nocc, 1), dtype=np.int32)
    kind = np.zeros(max(nc, 1), dtype=np.uint8)
    table = np.zeros(max(ntab, 1), dtype=np.uint32)
    opens = np.zeros(max(nopen, 1), dtype=np.int32)
    _check(lib().tnc_network_formula(net.h, *[ctypes.byref(x) for x in a], _p(arity, ctypes.c_int32),
                                     _p(var_of, ctypes.c_int32), _p(kind, ctypes.c_uint8), _p(table, ctypes.c_uint32),
                                     _p(opens, ctypes.c_int32)))
    clauses, kinds, tables, o, t = [], [], [], 0, 0
    for c in range(nc):
        clauses.append(tuple(int(v) for v in var_of[o:o + arity[c]]))
        o += int(arity[c])
        kinds.append(int(kind[c]))
        if kind[c] == 3:
            tables.append([int(x) for x in table[t:t + (1 << int(arity[c]))]])
            t += 1 << int(arity[c])
        else:
            tables.append(None)
    return FormulaView(nv, clauses, kinds, tables, [int(v) for v in opens[:nopen]])


def slice_network(formula, fixed: dict) -> FormulaView:
    """tnc_slice_network: the formula of the slice with the variables of
    `fixed` set to their values (read back through tnc_network_formula)."""
    net = build_network(formula)
    vs = list(fixed)
    bits = sum((int(fixed[v]) & 1) << i for i, v in enumerate(vs))
    arr = np.array(vs or [0], dtype=np.int32)
    h = ctypes.c_void_p()
    _check(lib().tnc_slice_network(net.h, len(vs), _p(arr, ctypes.c_int32), bits, ctypes.byref(h)))
    return network_formula(Network(h))


def plan_formula(formula, **kw) -> Plan:
    net = build_network(formula)
    return plan(net, n_open=len(formula.open_vars), **kw)


# ------------------------------------------------------------------ contraction

@dataclass
class Count:
    counts: List[int]          # exact CRT values, one per open index
    residues: np.ndarray       # [n_out, R]
    primes: List[int]
    flags: int

    @property
    def value(self) -> int:
        return self.counts[0]


def _opts(n_residues: int, primes: Optional[Sequence[int]], path: str = "int64"):
    pr = np.array(list(primes) if primes is not None else default_primes(n_residues, path), dtype=np.uint32)
    o = _ContractOpts(PATHS[path], n_residues, _p(pr, ctypes.c_uint32))
    return o, pr


def _count_buffers(n_out: int, R: int):
    res = np.zeros((n_out, R), dtype=np.uint32)
    cap_limbs = (31 * R + 31) // 32
    limbs = np.zeros((n_out, cap_limbs), dtype=np.uint32)
    c = _Count(_p(res, ctypes.c_uint32), _p(limbs, ctypes.c_uint32), n_out, cap_limbs, 0, 0, 0)
    return c, res, limbs


def _to_count(c: _Count, res: np.ndarray, limbs: np.ndarray, primes) -> Count:
    counts = []
    for row in limbs[: c.n_out]:
        v = 0
        for x in row[::-1]:
            v = (v << 32) | int(x)
        counts.append(v)
    return Count(counts, res[: c.n_out].copy(), [int(p) for p in primes], int(c.flags))


def _stream_ptr(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, ws=None):
    import torch
    if ws is not None:
        if ws.numel() * ws.element_size() < nbytes:
            raise ValueError("workspace too small")
        return ws
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")


def workspace_bytes(p: Plan, n_residues: int, path: str = "int64", primes=None) -> int:
    """tnc_workspace_bytes_opts for the path (tnc_workspace_bytes on int64 / tc)."""
    o, _ = _opts(n_residues, primes, path)
    nb = int(lib().tnc_workspace_bytes_opts(p.h, ctypes.byref(o)))
    if nb == 0:
        raise TncError(-1, lib().tnc_last_error().decode() or "invalid contract options")
    return nb


def contract(p: Plan, n_residues: int = 4, primes=None, workspace=None, stream=None, path: str = "int64") -> Count:
    """Contract one plan on the GPU (tnc_contract); returns exact counts."""
    o, pr = _opts(n_residues, primes, path)
    nb = workspace_bytes(p, n_residues, path, primes)
    ws = _workspace(nb, workspace)
    c, res, limbs = _count_buffers(1 << p.n_open, n_residues)
    _check(lib().tnc_contract(p.h, ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), nb, _stream_ptr(stream),
                              ctypes.byref(c)))
    return _to_count(c, res, limbs, pr)


def workspace_bytes_many(plans: Sequence[Plan], n_residues: int, path: str = "int64", group: int = 1,
                         primes=None) -> int:
    """tnc_workspace_bytes_many: bytes for groups of `group` consecutive plans."""
    o, _ = _opts(n_residues, primes, path)
    arr = (ctypes.c_void_p * len(plans))(*[pp.h.value for pp in plans])
    nb = int(lib().tnc_workspace_bytes_many(arr, len(plans), ctypes.byref(o), group))
    if nb == 0:
        raise TncError(-1, lib().tnc_last_error().decode() or "invalid arguments")
    return nb


def contract_many(plans: Sequence[Plan], n_residues: int = 4, primes=None, workspace=None, stream=None,
                  path: str = "int64", group: int = 16) -> List[Count]:
    """tnc_contract_many: many plans, tree levels merged within groups that
    fit the workspace (default: a workspace for groups of `group` plans)."""
    o, pr = _opts(n_residues, primes, path)
    arr = (ctypes.c_void_p * len(plans))(*[pp.h.value for pp in plans])
    nb = workspace_bytes_many(plans, n_residues, path, group, primes) if workspace is None else \
        workspace.numel() * workspace.element_size()
    ws = _workspace(nb, workspace)
    bufs = [_count_buffers(1 << pp.n_open, n_residues) for pp in plans]
    outs = (_Count * len(plans))(*[b[0] for b in bufs])
    _check(lib().tnc_contract_many(arr, len(plans), ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), nb,
                                   _stream_ptr(stream), outs))
    return [_to_count(outs[i], bufs[i][1], bufs[i][2], pr) for i in range(len(plans))]


def set_step_timing(on: bool):
    """tnc_set_step_timing: time every dense step of later contractions (this thread)."""
    lib().tnc_set_step_timing(1 if on else 0)


def last_dense_time() -> Tuple[float, int]:
    """tnc_last_dense_time: (device ms of the dense steps, their count) of the last contraction."""
    ms, n = ctypes.c_double(), ctypes.c_int32()
    _check(lib().tnc_last_dense_time(ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


def last_contract_time() -> float:
    """tnc_last_contract_time: device ms of the last contraction's kernels (timing mode)."""
    ms = ctypes.c_double()
    _check(lib().tnc_last_contract_time(ctypes.byref(ms)))
    return ms.value


P8_TILE_WIDTHS = (16, 32, 64, 128, 256)


def last_launch_counts() -> dict:
    """tnc_last_launch_counts: kernels the calling thread's last contraction
    enqueued, by kind; "p8_tile_n" maps tile width -> GEMM launches."""
    c = _LaunchCounts()
    _check(lib().tnc_last_launch_counts(ctypes.byref(c)))
    d = {n: int(getattr(c, n)) for n, _ in _LaunchCounts._fields_ if n != "p8_tile_n"}
    d["p8_tile_n"] = {w: int(c.p8_tile_n[i]) for i, w in enumerate(P8_TILE_WIDTHS)}
    return d


def last_dense_steps() -> List[dict]:
    """tnc_last_dense_steps: per dense launch of the last contraction (timing
    mode): ms, macs per residue, operand free bits, shared bits, residues,
    tile width, K split."""
    n = ctypes.c_int32()
    _check(lib().tnc_last_dense_steps(None, 0, ctypes.byref(n)))
    arr = (_DenseStepTime * max(n.value, 1))()
    _check(lib().tnc_last_dense_steps(arr, n.value, ctypes.byref(n)))
    return [{f: getattr(arr[i], f) for f, _ in _DenseStepTime._fields_} for i in range(n.value)]


def last_io_bytes() -> Tuple[int, int]:
    """tnc_last_io_bytes: (host->device, device->host) bytes of the last contraction."""
    a, b = ctypes.c_uint64(), ctypes.c_uint64()
    _check(lib().tnc_last_io_bytes(ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def contract_sliced(plans: Sequence[Plan], n_residues: int = 4, primes=None, workspace=None, stream=None,
                    path: str = "int64") -> Count:
    """tnc_contract_sliced: the sum of the plans' counts (the slices of one
    formula), added as residues on the device, one CRT."""
    o, pr = _opts(n_residues, primes, path)
    arr = (ctypes.c_void_p * len(plans))(*[pp.h.value for pp in plans])
    nb = int(lib().tnc_workspace_bytes_sliced(arr, len(plans), ctypes.byref(o)))
    if nb == 0:
        raise TncError(-1, lib().tnc_last_error().decode() or "invalid slices")
    ws = _workspace(nb, workspace)
    nb = ws.numel() * ws.element_size()  # a larger workspace lets slices run merged
    c, res, limbs = _count_buffers(1 << plans[0].n_open, n_residues)
    _check(lib().tnc_contract_sliced(arr, len(plans), ctypes.byref(o), ctypes.c_void_p(ws.data_ptr()), nb,
                                     _stream_ptr(stream), ctypes.byref(c)))
    return _to_count(c, res, limbs, pr)


def crt_host(primes: Sequence[int], residues) -> List[int]:
    """tnc_crt_host: exact values in [0, prod p) from residues [n, R] (host)."""
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    res = np.ascontiguousarray(np.asarray(residues, dtype=np.uint32).reshape(-1, len(pr)))
    need = ctypes.c_int32()
    cap = int(sum(np.log2(pr.astype(np.float64))) // 32) + 1
    limbs = np.zeros((max(res.shape[0], 1), cap), dtype=np.uint32)
    _check(lib().tnc_crt_host(_p(pr, ctypes.c_uint32), len(pr), _p(res, ctypes.c_uint32), res.shape[0],
                              _p(limbs, ctypes.c_uint32), cap, ctypes.byref(need)))
    return Batch.counts_from_limbs(limbs[: res.shape[0]])


def residue_add_host(primes: Sequence[int], acc: np.ndarray, src: np.ndarray) -> np.ndarray:
    """tnc_residue_add_host: acc = (acc + src) mod primes, residue by residue (in place)."""
    pr = np.ascontiguousarray(np.asarray(primes, dtype=np.uint32))
    assert acc.dtype == np.uint32 and acc.flags.c_contiguous and acc.shape == src.shape
    s = np.ascontiguousarray(src, dtype=np.uint32)
    _check(lib().tnc_residue_add_host(_p(pr, ctypes.c_uint32), len(pr), _p(acc, ctypes.c_uint32),
                                      _p(s, ctypes.c_uint32), acc.size // len(pr)))
    return acc


def probe_modmac(iters: int = 4096, stream=None) -> float:
    """Measured modular MAC/s of the step kernels' inner primitive (tnc_probe_modmac)."""
    v = ctypes.c_double()
    _check(lib().tnc_probe_modmac(_stream_ptr(stream), iters, ctypes.byref(v)))
    return v.value


def contract_noalloc(p: Plan, n_residues: int = 4, primes=None, stream=None, path: str = "int64") -> Count:
    """tnc_contract_noalloc: like contract(), but the device scratch is libtnc's
    own fixed array, so nothing is allocated on the device for the call (for
    callers that cannot allocate device memory; see include/tnc.h)."""
    o, pr = _opts(n_residues, primes, path)
    c, res, limbs = _count_buffers(1 << p.n_open, n_residues)
    _check(lib().tnc_contract_noalloc(p.h, ctypes.byref(o), _stream_ptr(stream), ctypes.byref(c)))
    return _to_count(c, res, limbs, pr)


class Batch:
    """tnc_batch_t: many plans in one persistent, graph-captured launch."""

    def __init__(self, plans: Sequence[Plan], n_residues: int = 2, primes=None, path: str = "int64"):
        self.plans = list(plans)
        self.R = n_residues
        self._o, self._pr = _opts(n_residues, primes, path)
        arr = (ctypes.c_void_p * len(self.plans))(*[pp.h.value for pp in self.plans])
        self._arr = arr
        h = ctypes.c_void_p()
        _check(lib().tnc_batch_create(arr, len(self.plans), ctypes.byref(self._o), ctypes.byref(h)))
        self.h = h

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tnc_free_batch(self.h)
            self.h = None

    def workspace_bytes(self) -> int:
        return int(lib().tnc_batch_workspace_bytes(self.h))

    def info(self):
        """(h2d bytes per upload, d2h bytes per download, result entries, kernels per launch)."""
        a, b, c, d = ctypes.c_size_t(), ctypes.c_size_t(), ctypes.c_uint64(), ctypes.c_int32()
        _check(lib().tnc_batch_info(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
        return a.value, b.value, c.value, d.value

    def upload(self, ws, stream=None):
        _check(lib().tnc_batch_upload(self.h, ctypes.c_void_p(ws.data_ptr()), self.workspace_bytes(),
                                      _stream_ptr(stream)))

    def launch(self, ws, stream=None):
        _check(lib().tnc_batch_launch(self.h, ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream)))

    def autotune(self, ws, stream=None) -> Tuple[int, int, int]:
        """tnc_batch_autotune: returns (threads per CTA, shared-memory arena
        bytes, CTAs-per-SM cap with 0 = as many as fit)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tnc_batch_autotune(self.h, ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream),
                                        ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def set_launch(self, threads: int, smem_bytes: int, ctas_per_sm: int = 0):
        """tnc_batch_set_launch: fix the launch shape without timing."""
        _check(lib().tnc_batch_set_launch(self.h, int(threads), int(smem_bytes), int(ctas_per_sm)))

    def get_launch(self) -> Tuple[int, int, int]:
        """tnc_batch_get_launch: (threads, shared-memory arena bytes, CTAs-per-SM cap)."""
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tnc_batch_get_launch(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
        return a.value, b.value, c.value

    def signature(self) -> str:
        """What an autotuned launch shape depends on: the device and the
        batch's sizes (descriptor bytes, result entries, formulas, residues)."""
        import torch
        h2d, _, n_entries, _ = self.info()
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        return f"{props.name}|{props.multi_processor_count}|{h2d}|{n_entries}|{len(self.plans)}|{self.R}"

    def autotune_cached(self, ws, stream=None, cache: Optional[str] = None) -> Tuple[int, int, int]:
        """The launch shape from the JSON file `cache` if it holds one for this
        batch's signature (tnc_batch_set_launch, no timing); else
        tnc_batch_autotune, whose choice is then added to the file."""
        import json
        key = self.signature()
        table = {}
        if cache and os.path.exists(cache):
            with open(cache) as fh:
                table = json.load(fh)
        if key in table:
            self.set_launch(*table[key])
            return tuple(table[key])
        shape = self.autotune(ws, stream)
        if cache:
            table[key] = list(shape)
            tmp = f"{cache}.tmp{os.getpid()}"
            with open(tmp, "w") as fh:
                json.dump(table, fh, indent=1)
            os.replace(tmp, cache)
        return shape

    def download(self, ws, stream=None) -> List[Count]:
        n = len(self.plans)
        bufs = [_count_buffers(1 << pp.n_open, self.R) for pp in self.plans]
        arr = (_Count * n)(*[b[0] for b in bufs])
        _check(lib().tnc_batch_download(self.h, ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream), arr))
        return [_to_count(arr[i], bufs[i][1], bufs[i][2], self._pr) for i in range(n)]

    def download_flat(self, ws, stream=None, out=None):
        """tnc_batch_download_flat into reusable numpy arrays:
        (residues [E, R], limbs [E, L], flags [n]); entries formula after formula."""
        _, _, n_entries, _ = self.info()
        L = (31 * self.R + 31) // 32
        if out is None:
            out = (np.empty((n_entries, self.R), dtype=np.uint32), np.empty((n_entries, L), dtype=np.uint32),
                   np.empty(len(self.plans), dtype=np.uint32))
        res, limbs, flags = out
        _check(lib().tnc_batch_download_flat(self.h, ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream),
                                             _p(res, ctypes.c_uint32), _p(limbs, ctypes.c_uint32),
                                             _p(flags, ctypes.c_uint32)))
        return out

    @staticmethod
    def counts_from_limbs(limbs: np.ndarray) -> List[int]:
        out = []
        for row in limbs:
            v = 0
            for x in row[::-1]:
                v = (v << 32) | int(x)
            out.append(v)
        return out

    def status(self, ws, stream=None) -> int:
        return int(lib().tnc_batch_status(self.h, ctypes.c_void_p(ws.data_ptr()), _stream_ptr(stream)))


def contract_batch(plans: Sequence[Plan], n_residues: int = 2, primes=None, workspace=None, stream=None,
                   path: str = "int64") -> List[Count]:
    """Upload + persistent launch + download (tnc_contract_batch)."""
    b = Batch(plans, n_residues, primes, path)
    ws = _workspace(b.workspace_bytes(), workspace)
    n = len(b.plans)
    bufs = [_count_buffers(1 << pp.n_open, n_residues) for pp in b.plans]
    arr = (_Count * n)(*[x[0] for x in bufs])
    _check(lib().tnc_contract_batch(b._arr, n, ctypes.byref(b._o), ctypes.c_void_p(ws.data_ptr()),
                                    b.workspace_bytes(), _stream_ptr(stream), arr))
    return [_to_count(arr[i], bufs[i][1], bufs[i][2], b._pr) for i in range(n)]


def count(formula, n_residues: int = 4, heuristic: str = "bisect", **kw) -> Count:
    """Convenience: build, plan and contract one formula."""
    return contract(plan_formula(formula, heuristic=heuristic), n_residues, **kw)


# ------------------------------------------------------------------ learned ordering

def _dp(x):
    return ctypes.c_void_p(x.data_ptr() if x is not None else 0)


def inject_failure(kind: str, after: int = 0):
    """tnc_inject_failure: arm one host-side failure ("nomem", "plan",
    "launch", "timeout"; "none" disarms)."""
    _check(lib().tnc_inject_failure(INJECT[kind], after))


def learned_save(path: str, params: np.ndarray):
    """tnc_learned_save: host fp32 scorer parameters to a checked file."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    assert p.size == MLP_PARAMS
    _check(lib().tnc_learned_save(path.encode(), _p(p, ctypes.c_float)))


def learned_load(path: str) -> np.ndarray:
    """tnc_learned_load: the parameters of a file written by learned_save."""
    out = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(lib().tnc_learned_load(path.encode(), _p(out, ctypes.c_float)))
    return out


def mlp_init(seed: int = 0) -> np.ndarray:
    """He-initialised scorer parameters (fp32, TNC_MLP_PARAMS)."""
    out = np.zeros(MLP_PARAMS, dtype=np.float32)
    _check(lib().tnc_mlp_init(seed, _p(out, ctypes.c_float)))
    return out


def learned_dataset(formulas, states: int = 2, cands: int = 16, seed: int = 0):
    """(X [rows, 16], T [rows]) float32: features and rollout regrets."""
    nets = [build_network(f) for f in formulas]
    arr = (ctypes.c_void_p * len(nets))(*[x.h.value for x in nets])
    n = ctypes.c_int64()
    rc = lib().tnc_learned_dataset(arr, len(nets), states, cands, seed, None, None, 0, ctypes.byref(n))
    if rc not in (TNC_OK, -4):
        _check(rc)
    X = np.zeros((max(n.value, 1), MLP_FEATURES), dtype=np.float32)
    T = np.zeros(max(n.value, 1), dtype=np.float32)
    _check(lib().tnc_learned_dataset(arr, len(nets), states, cands, seed, _p(X, ctypes.c_float),
                                     _p(T, ctypes.c_float), n.value, ctypes.byref(n)))
    return X[: n.value], T[: n.value]


def learned_dataset_on_policy(formulas, params_bf16, states: int = 2, seed: int = 0, stream=None):
    """Rows along the learned planner's own trajectories (second training round)."""
    import torch
    nets = [build_network(f) for f in formulas]
    n = len(nets)
    arr = (ctypes.c_void_p * n)(*[x.h.value for x in nets])
    ws = torch.empty(int(lib().tnc_plan_learned_workspace_bytes(n)), dtype=torch.uint8, device=params_bf16.device)
    cnt = ctypes.c_int64()
    rc = lib().tnc_learned_dataset_on_policy(arr, n, _dp(params_bf16), _dp(ws), ws.numel(), _stream_ptr(stream),
                                             states, seed, None, None, 0, ctypes.byref(cnt))
    if rc not in (TNC_OK, -4):
        _check(rc)
    X = np.zeros((max(cnt.value, 1), MLP_FEATURES), dtype=np.float32)
    T = np.zeros(max(cnt.value, 1), dtype=np.float32)
    _check(lib().tnc_learned_dataset_on_policy(arr, n, _dp(params_bf16), _dp(ws), ws.numel(), _stream_ptr(stream),
                                               states, seed, _p(X, ctypes.c_float), _p(T, ctypes.c_float),
                                               cnt.value, ctypes.byref(cnt)))
    return X[: cnt.value], T[: cnt.value]


def mlp_forward(params, x, y, h1=None, h2=None, stream=None):
    """Device tensors (torch): params [P] f32, x [rows,16] f32 -> y [rows]."""
    _check(lib().tnc_mlp_forward(_dp(params), _dp(x), x.shape[0], _dp(y), _dp(h1), _dp(h2), _stream_ptr(stream)))


def mlp_backward(params, x, h1, h2, y, t, grads, stream=None):
    import torch
    scratch = torch.empty(int(lib().tnc_mlp_backward_scratch_floats(x.shape[0])) + 1, dtype=torch.float32,
                          device=x.device)
    _check(lib().tnc_mlp_backward(_dp(params), _dp(x), _dp(h1), _dp(h2), _dp(y), _dp(t), x.shape[0], _dp(scratch),
                                  _dp(grads), _stream_ptr(stream)))


def mlp_adam(params, grads, m, v, step: int, lr: float, stream=None):
    _check(lib().tnc_mlp_adam(_dp(params), _dp(grads), _dp(m), _dp(v), step, lr, _stream_ptr(stream)))


def mlp_train(params, x, t, epochs: int = 20, batch: int = 4096, lr: float = 1e-3, stream=None) -> List[float]:
    """Train in place on device rows; returns per-epoch mean squared error."""
    import torch
    ws = torch.empty(int(lib().tnc_mlp_train_workspace_bytes(batch)), dtype=torch.uint8, device=x.device)
    loss = (ctypes.c_float * epochs)()
    _check(lib().tnc_mlp_train(_dp(params), _dp(x), _dp(t), x.shape[0], epochs, batch, lr, _dp(ws), ws.numel(),
                               _stream_ptr(stream), loss))
    return [float(v) for v in loss]


def mlp_to_bf16(params, out, stream=None):
    _check(lib().tnc_mlp_to_bf16(_dp(params), _dp(out), _stream_ptr(stream)))


def mlp_forward_bf16(params_bf16, x, y, stream=None):
    _check(lib().tnc_mlp_forward_bf16(_dp(params_bf16), _dp(x), x.shape[0], _dp(y), _stream_ptr(stream)))


def plan_learned_many(formulas, params_bf16, fallback: str = "best", rank_cap: int = 32, stream=None):
    """Learned plans with heuristic fallback.  Returns (plans, chose_learned
    list, learned_macs list)."""
    import torch
    nets = [build_network(f) for f in formulas]
    n = len(nets)
    arr = (ctypes.c_void_p * n)(*[x.h.value for x in nets])
    outs = (ctypes.c_void_p * n)()
    sts = (_PlanStats * n)()
    chose = np.zeros(n, dtype=np.int32)
    lmacs = np.zeros(n, dtype=np.float64)
    ordr = np.zeros(1, dtype=np.int32)
    o = _PlanOpts(HEURISTICS[fallback], rank_cap, 2, 0, _p(ordr, ctypes.c_int32), 0)
    ws = torch.empty(int(lib().tnc_plan_learned_workspace_bytes(n)), dtype=torch.uint8, device=params_bf16.device)
    _check(lib().tnc_plan_learned_many(arr, n, _dp(params_bf16), ctypes.byref(o), _dp(ws), ws.numel(),
                                       _stream_ptr(stream), outs, sts, _p(chose, ctypes.c_int32),
                                       _p(lmacs, ctypes.c_double)))
    plans = [Plan(ctypes.c_void_p(outs[i]), _stats(sts[i]), len(formulas[i].open_vars)) for i in range(n)]
    return plans, chose.tolist(), lmacs.tolist()


def _learned_opts(states=2, cands=8, completion="best", checkpoints=(), max_pct=100, seed=0):
    cp = list(checkpoints)[:8]
    arr = (ctypes.c_int32 * 8)(*(cp + [0] * (8 - len(cp))))
    return _LearnedOpts(states, cands, HEURISTICS[completion], len(cp), arr, max_pct, seed)


def plan_learned_coarsen(formulas, params_bf16=None, completion: str = "best",
                         checkpoints: Sequence[int] = (20, 35, 50, 65, 80), fallback: str = "best",
                         rank_cap: int = 64, seed: int = 0, stream=None):
    """tnc_plan_learned_opts: learned merges coarsen each network, the
    heuristic `completion` finishes it at each checkpoint (% of the merges),
    the cheapest is the learned plan, kept only if not worse than `fallback`.
    params_bf16 None: tensor-greedy coarsening (no scorer, host only).
    Returns (plans, chose_learned list, learned_macs list)."""
    nets = [build_network(f) for f in formulas]
    n = len(nets)
    arr = (ctypes.c_void_p * n)(*[x.h.value for x in nets])
    outs = (ctypes.c_void_p * n)()
    sts = (_PlanStats * n)()
    chose = np.zeros(n, dtype=np.int32)
    lmacs = np.zeros(n, dtype=np.float64)
    ordr = np.zeros(1, dtype=np.int32)
    fb = _PlanOpts(HEURISTICS[fallback], rank_cap, 2, 0, _p(ordr, ctypes.c_int32), 0)
    lo = _learned_opts(completion=completion, checkpoints=checkpoints, seed=seed)
    ws, nb = None, 0
    if params_bf16 is not None:
        import torch
        ws = torch.empty(int(lib().tnc_plan_learned_workspace_bytes(n)), dtype=torch.uint8, device=params_bf16.device)
        nb = ws.numel()
    _check(lib().tnc_plan_learned_opts(arr, n, _dp(params_bf16), ctypes.byref(lo), ctypes.byref(fb), _dp(ws), nb,
                                       _stream_ptr(stream) if params_bf16 is not None else None, outs, sts,
                                       _p(chose, ctypes.c_int32), _p(lmacs, ctypes.c_double)))
    plans = [Plan(ctypes.c_void_p(outs[i]), _stats(sts[i]), len(formulas[i].open_vars)) for i in range(n)]
    return plans, chose.tolist(), lmacs.tolist()


def learned_dataset_coarsen(formulas, states: int = 2, cands: int = 8, completion: str = "best", max_pct: int = 80,
                            seed: int = 0, params_bf16=None, stream=None):
    """tnc_learned_dataset_opts: rows labelled by heuristic completion
    ((X [rows, 16], T [rows]) float32)."""
    nets = [build_network(f) for f in formulas]
    n = len(nets)
    arr = (ctypes.c_void_p * n)(*[x.h.value for x in nets])
    lo = _learned_opts(states=states, cands=cands, completion=completion, max_pct=max_pct, seed=seed)
    ws, nb = None, 0
    if params_bf16 is not None:
        import torch
        ws = torch.empty(int(lib().tnc_plan_learned_workspace_bytes(n)), dtype=torch.uint8, device=params_bf16.device)
        nb = ws.numel()
    st = _stream_ptr(stream) if params_bf16 is not None else None
    cnt = ctypes.c_int64()
    rc = lib().tnc_learned_dataset_opts(arr, n, ctypes.byref(lo), _dp(params_bf16), _dp(ws), nb, st, None, None, 0,
                                        ctypes.byref(cnt))
    if rc not in (TNC_OK, -4):
        _check(rc)
    X = np.zeros((max(cnt.value, 1), MLP_FEATURES), dtype=np.float32)
    T = np.zeros(max(cnt.value, 1), dtype=np.float32)
    _check(lib().tnc_learned_dataset_opts(arr, n, ctypes.byref(lo), _dp(params_bf16), _dp(ws), nb, st,
                                          _p(X, ctypes.c_float), _p(T, ctypes.c_float), cnt.value, ctypes.byref(cnt)))
    return X[: cnt.value], T[: cnt.value]
