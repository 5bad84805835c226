"""Build libotfmm.so in-tree for sm_103a with nvcc.

``python -m paper_2303_08058_b300.build`` (or ``build()``) regenerates the
contraction code if its generator changed, then compiles the kernels and the
host library into ``paper_2303_08058_b300/libotfmm.so``.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libotfmm.so")
SOURCES = [os.path.join(CSRC, f) for f in ("ot_kernels.cu", "ot_lib.cu", "ot_noalloc.cu")]
DEPS = SOURCES + [os.path.join(CSRC, f) for f in ("ot_internal.h", "ot_contract.inc", "ot_contract_counts.h",
                                                  "gen_contract.py")] + \
    [os.path.join(ROOT, "include", "ot.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force: bool = False, verbose: bool = False) -> str:
    inc = os.path.join(CSRC, "ot_contract.inc")
    gen = os.path.join(CSRC, "gen_contract.py")
    counts = os.path.join(CSRC, "ot_contract_counts.h")
    if force or _stale(inc, [gen]) or _stale(counts, [gen]):
        subprocess.run([sys.executable, gen], check=True)
    if not (force or _stale(LIB, DEPS)):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-o", tmp, *SOURCES, "-lcudart"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd))
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
