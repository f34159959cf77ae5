"""Builds the in-tree CUDA library ``libqaoa_b300.so`` for sm_103a with nvcc.

``python -m paper_2312_03019_b300.build [--force] [--verbose] [--debug-bounds]``; the shared
object lands next to this file, so it travels with the source tree.  Units compile in parallel
into ``_build/`` (git-ignored) and only stale ones are recompiled; ``--force`` recompiles all,
``--verbose`` recompiles all with ``-Xptxas -v`` (registers, spills, shared memory per kernel).
``--debug-bounds`` builds ``libqaoa_b300_debug.so`` instead, with the kernels' index checks
compiled in (-DQAOA_DEBUG_BOUNDS; see qaoa_debug_bounds_read); the binding loads it when the
environment variable QAOA_LIBRARY names it.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libqaoa_b300.so")
LIB_DEBUG = os.path.join(HERE, "libqaoa_b300_debug.so")
# translation units, compiled in parallel and linked into one shared object
SOURCES = ["capi.cu", "tile_c64.cu", "recipes_c64.cu", "recipes_w_c64.cu", "tile_c128.cu", "grad_kernels.cu",
           "grad_recipes.cu", "grad_recipes_m.cu", "grad_recipes_x.cu", "grad_pf.cu", "grad_pf_w.cu", "recipes2_c64.cu", "batch_c64.cu", "plan.cpp"]
HEADERS = ["kernels.cuh", "plan.h", "server.cuh", "instances.h", os.path.join("..", "..", "include", "qaoa.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = SOURCES + HEADERS + [os.path.basename(__file__)]
    for d in deps:
        p = os.path.join(CSRC, d) if not d.endswith("build.py") else os.path.join(HERE, d)
        if os.path.exists(p) and os.path.getmtime(p) > t:
            return True
    return False


def _dep_time() -> float:
    """Newest modification time among the headers and this script (they affect every unit)."""
    t = os.path.getmtime(os.path.abspath(__file__))
    for h in HEADERS:
        p = os.path.join(CSRC, h)
        if os.path.exists(p):
            t = max(t, os.path.getmtime(p))
    return t


def build(force: bool = False, verbose: bool = False, debug_bounds: bool = False) -> str:
    lib = LIB_DEBUG if debug_bounds else LIB
    if not (force or verbose or _stale(lib)):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    # kernel template instances live in their own units: their host stubs need external linkage
    flags = ["-O3", "-std=c++17", *ARCH, "-lineinfo", "-static-global-template-stub=false", "-Xcompiler",
             "-fPIC,-O2"]
    if verbose:
        flags += ["-Xptxas", "-v"]
    extra = os.environ.get("QAOA_NVCC_EXTRA", "").split()
    flags += extra
    if debug_bounds:
        flags += ["-DQAOA_DEBUG_BOUNDS"]
    # objects are kept (per flag set) so that a change to one unit recompiles only that unit
    objdir = os.path.join(HERE, "_build", "debug" if debug_bounds else ("extra" if extra else "default"))
    os.makedirs(objdir, exist_ok=True)
    dep_t = _dep_time()
    objs, procs = [], []
    for src in SOURCES:
        srcp = os.path.join(CSRC, src)
        obj = os.path.join(objdir, src + ".o")
        objs.append(obj)
        fresh = os.path.exists(obj) and os.path.getmtime(obj) >= max(dep_t, os.path.getmtime(srcp))
        if fresh and not (force or verbose or extra):
            continue
        procs.append((obj, subprocess.Popen([nvcc, *flags, "-c", srcp, "-o", obj + ".tmp"],
                                            stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
    failed = False
    for obj, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            failed = True
            sys.stderr.write(out)
            continue
        os.replace(obj + ".tmp", obj)
        if verbose:
            sys.stderr.write(out)
    if failed:
        raise RuntimeError("nvcc failed building libqaoa_b300.so")
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", lib + ".tmp", *objs], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError(f"nvcc failed linking {os.path.basename(lib)}")
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="--verbose" in sys.argv,
                debug_bounds="--debug-bounds" in sys.argv))
