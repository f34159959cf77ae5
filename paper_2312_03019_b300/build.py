"""Builds the in-tree CUDA library ``libqaoa_b300.so`` for sm_103a with nvcc.

``python -m paper_2312_03019_b300.build [--verbose]``; the shared object lands next to this
file, so it travels with the source tree.  ``--verbose`` adds ``-Xptxas -v`` (registers,
spills, shared memory per kernel).
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libqaoa_b300.so")
SOURCES = ["capi.cu", "plan.cpp"]
HEADERS = ["kernels.cuh", "plan.h", "server.cuh", os.path.join("..", "..", "include", "qaoa.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + HEADERS + [os.path.basename(__file__)]
    for d in deps:
        p = os.path.join(CSRC, d) if not d.endswith("build.py") else os.path.join(HERE, d)
        if os.path.exists(p) and os.path.getmtime(p) > t:
            return True
    return False


def build(force: bool = False, verbose: bool = False) -> str:
    if not (force or verbose or _stale()):
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O2", "-shared",
           "-o", LIB + ".tmp"] + [os.path.join(CSRC, s) for s in SOURCES]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += os.environ.get("QAOA_NVCC_EXTRA", "").split()
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed building libqaoa_b300.so")
    if verbose:
        sys.stderr.write(r.stderr)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose="--verbose" in sys.argv)
    print(LIB)
