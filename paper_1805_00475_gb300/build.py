"""Builds libtnc.so in-tree for sm_103a (nvcc + g++, no cmake).

    python -m paper_1805_00475_gb300.build [--force]

Host sources (planner, lowering, ABI) compile with g++; CUDA sources with nvcc
for `-gencode arch=compute_103a,code=sm_103a`; everything is linked by nvcc
into paper_1805_00475_gb300/_lib/libtnc.so with the static CUDA runtime.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libtnc.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SRC = ["network.cpp", "planner.cpp", "lower.cpp", "learned.cpp", "slicing.cpp", "combine.cpp", "inject.cpp", "abi_host.cpp"]
CUDA_SRC = ["contract.cu", "probe.cu", "tc.cu", "tc_p8.cu", "mlp.cu"]
HEADERS = ["tnc_internal.h", "step_desc.h", "kernels.cuh", "modarith.cuh"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtnc")


def _newest(paths) -> float:
    return max(os.path.getmtime(p) for p in paths)


def _commands():
    nvcc = _nvcc()
    inc = ["-I", INCLUDE, "-I", CSRC]
    cmds = []
    for s in HOST_SRC:
        o = os.path.join(OBJ, s + ".o")
        cmds.append((o, os.path.join(CSRC, s),
                     ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-fopenmp", *inc, "-c",
                      os.path.join(CSRC, s), "-o", o]))
    for s in CUDA_SRC:
        o = os.path.join(OBJ, s + ".o")
        cmds.append((o, os.path.join(CSRC, s),
                     [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC",
                      "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, s), "-o", o]))
    return nvcc, cmds


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc, cmds = _commands()
    deps = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(INCLUDE, "tnc.h")]
    hdr_time = _newest(deps)
    todo = [c for c in cmds if force or not os.path.exists(c[0])
            or os.path.getmtime(c[0]) < max(os.path.getmtime(c[1]), hdr_time)]

    def run(c):
        if verbose:
            print(" ".join(c[2]), flush=True)
        r = subprocess.run(c[2], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(c[2])}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
        for msg in ex.map(run, todo):
            if verbose and msg:
                print(msg)
    objs = [c[0] for c in cmds]
    if force or todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < _newest(objs):
        tmp = LIB + f".tmp{os.getpid()}"
        link = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
        r = subprocess.run(link, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed: {' '.join(link)}\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
