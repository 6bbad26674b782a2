"""Exact CPU oracle for tensor-network model counting -- TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline/reference leg
may import this package.  The product path (the CUDA library and its Python
binding) never does, and this package imports nothing from the product: it
reads formulas as plain attributes (n_vars, clauses, kinds, tables,
open_vars), whoever made them.

Two implementations of the same definition, sharing no code with each other:
  * tnc_oracle.c   (C, fixed-width big integers, OpenMP): brute force over all
                   assignments and pairwise contraction of the paper's network;
  * pyoracle.py    (pure Python ints, small cases only): the same two routes.
Counts come back as Python ints; residues mod p are taken here, by the caller,
from the exact value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import List, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tnc_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libtnc_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-Wall", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            u32p = ctypes.POINTER(ctypes.c_uint32)
            u8p = ctypes.POINTER(ctypes.c_uint8)
            lib.tnco_limbs.argtypes = [ctypes.c_int, ctypes.c_int, i32p, u8p, u32p]
            lib.tnco_limbs.restype = ctypes.c_int
            lib.tnco_bruteforce.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, u8p, u32p,
                                            ctypes.c_int, i32p, ctypes.c_int, u32p]
            lib.tnco_bruteforce.restype = ctypes.c_int
            lib.tnco_contract.argtypes = [ctypes.c_int, ctypes.c_int, i32p, i32p, u8p, u32p,
                                          ctypes.c_int, i32p, i32p, ctypes.c_int, ctypes.c_int,
                                          ctypes.c_int, u32p, i32p]
            lib.tnco_contract.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


class _Flat:
    """The formula as contiguous C arrays (kept alive while the call runs)."""

    def __init__(self, f):
        self.n_vars = int(f.n_vars)
        self.n_cons = len(f.clauses)
        self.arity = np.array([len(c) for c in f.clauses] or [0], dtype=np.int32)
        self.var_of = np.array([v for c in f.clauses for v in c] or [0], dtype=np.int32)
        self.kind = np.array(list(f.kinds) or [0], dtype=np.uint8)
        tab: List[int] = []
        for k, t in zip(f.kinds, f.tables):
            if t is not None and k == 3:
                tab.extend(int(x) for x in t)
        self.table = np.array(tab or [0], dtype=np.uint32)
        self.open = np.array(list(f.open_vars) or [0], dtype=np.int32)
        self.n_open = len(f.open_vars)

    def args(self):
        return (self.n_vars, self.n_cons, _ptr(self.arity, ctypes.c_int32),
                _ptr(self.var_of, ctypes.c_int32), _ptr(self.kind, ctypes.c_uint8),
                _ptr(self.table, ctypes.c_uint32))


def _to_ints(buf: np.ndarray, W: int) -> List[int]:
    out = []
    for row in buf.reshape(-1, W):
        v = 0
        for i in range(W - 1, -1, -1):
            v = (v << 32) | int(row[i])
        out.append(v)
    return out


def limbs(f) -> int:
    fl = _Flat(f)
    lib = _load()
    return lib.tnco_limbs(fl.n_vars, fl.n_cons, _ptr(fl.arity, ctypes.c_int32),
                          _ptr(fl.kind, ctypes.c_uint8), _ptr(fl.table, ctypes.c_uint32))


def bruteforce(f) -> List[int]:
    """Counts by enumerating all 2^n assignments (n <= 34); one per open index."""
    fl = _Flat(f)
    lib = _load()
    W = limbs(f)
    out = np.zeros(((1 << fl.n_open) * W,), dtype=np.uint32)
    rc = lib.tnco_bruteforce(*fl.args(), fl.n_open, _ptr(fl.open, ctypes.c_int32), W,
                             _ptr(out, ctypes.c_uint32))
    if rc != 0:
        raise RuntimeError(f"oracle bruteforce failed ({rc})")
    return _to_ints(out, W)


def contract(f, order: Optional[Sequence[Tuple[int, int]]] = None, max_rank: int = 30
             ) -> Tuple[List[int], int, int]:
    """Exact counts by pairwise contraction of the paper's network.

    order: optional pairs of tensor ids (clause c -> c, variable v -> n_cons+v,
    i-th result -> n_cons+n_vars+i); the rest follows tensor-greedy.
    Returns (counts, max rank seen, contractions done)."""
    fl = _Flat(f)
    lib = _load()
    W = limbs(f)
    out = np.zeros(((1 << fl.n_open) * W,), dtype=np.uint32)
    pairs = np.array([x for p in (order or []) for x in p] or [0], dtype=np.int32)
    stats = np.zeros(2, dtype=np.int32)
    rc = lib.tnco_contract(*fl.args(), fl.n_open, _ptr(fl.open, ctypes.c_int32),
                           _ptr(pairs, ctypes.c_int32), len(order or []), max_rank, W,
                           _ptr(out, ctypes.c_uint32), _ptr(stats, ctypes.c_int32))
    if rc == -2:
        raise OverflowError("oracle: intermediate rank above max_rank")
    if rc != 0:
        raise RuntimeError(f"oracle contract failed ({rc})")
    return _to_ints(out, W), int(stats[0]), int(stats[1])


def count(f, order=None, max_rank: int = 30) -> List[int]:
    return contract(f, order, max_rank)[0]


def residues(values: Sequence[int], primes: Sequence[int]) -> List[List[int]]:
    """[entry][prime] residues of exact counts, for comparison with a device path."""
    return [[v % p for p in primes] for v in values]
