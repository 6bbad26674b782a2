"""The toolchain fact behind the tensor-core arithmetic: the 8-bit integer
form of tcgen05.mma (kind::i8) does not exist for sm_103a, so exact 8-bit
limbs run as fp16 kind::f16 MMAs with fp32 accumulation kept below 2^24.
Checked by compiling (no GPU needed): ptxas rejects kind::i8 for sm_103a and
accepts the same instruction for sm_100a."""
import os
import shutil
import subprocess
import tempfile

import pytest

SRC = r"""
#include <cstdint>
__global__ void k(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, int acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::KIND [%0], %1, %2, %3, p;\n\t}\n"
               :: "r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
"""


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    pytest.skip("nvcc not available")


def _compile(kind: str, arch: str):
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "k.cu")
        with open(src, "w") as f:
            f.write(SRC.replace("KIND", kind))
        return subprocess.run([_nvcc(), "-gencode", f"arch=compute_{arch},code=sm_{arch}", "-c", src,
                               "-o", os.path.join(d, "k.o")], capture_output=True, text=True)


def test_int8_tcgen05_is_not_available_on_sm_103a():
    r = _compile("i8", "103a")
    assert r.returncode != 0
    assert "kind::i8" in (r.stdout + r.stderr)
    assert _compile("i8", "100a").returncode == 0     # the same instruction exists on sm_100a
    assert _compile("f16", "103a").returncode == 0    # the form the library uses
