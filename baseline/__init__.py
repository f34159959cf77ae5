"""The paper's optimised CPU method (Opt_u of Table 2) as a timing baseline: ctypes wrapper of
``opt_u.c``.  Neither the oracle nor the GPU path; ``bench.py`` times it beside them and
``tests/test_baseline_opt_u.py`` checks it against the oracle.

Angles are in the paper's convention: gamma_paper = -gamma and beta_paper = 2 beta relative to
the library's psi_z <- exp(-i gamma C(z)) psi_z and RX(2 beta).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "opt_u.c")
_LIB = os.path.join(_HERE, "libopt_u.so")
_lib = None


def build(force: bool = False) -> str:
    """gcc -O3 with OpenMP; x86-64-v2 for the hardware popcount the method relies on."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O3", "-std=c11", "-march=x86-64-v2", "-fopenmp", "-fPIC", "-shared", "-Wall",
               "-Wextra", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.c_void_p
        i32p = ctypes.POINTER(ctypes.c_int32)
        L.optu_qaoa.argtypes = [ctypes.c_int, ctypes.c_int, i32p, ctypes.c_int, dp, dp, dp]
        L.optu_expectation.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, dp, dp]
        L.optu_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def threads() -> int:
    return lib().optu_threads()


def run(g, gamma, beta):
    """State after len(gamma) levels, library convention angles in, complex128 out."""
    gp = np.ascontiguousarray(-np.asarray(gamma, dtype=np.float64))
    bp = np.ascontiguousarray(2.0 * np.asarray(beta, dtype=np.float64))
    e = np.ascontiguousarray(np.asarray(g.edges, dtype=np.int32).reshape(-1))
    psi = np.empty(1 << g.n, dtype=np.complex128)
    rc = lib().optu_qaoa(g.n, g.m, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), len(gp),
                         ctypes.c_void_p(gp.ctypes.data), ctypes.c_void_p(bp.ctypes.data),
                         ctypes.c_void_p(psi.ctypes.data))
    if rc:
        raise ValueError("opt_u rejected the graph")
    return psi


def expectation(g, psi):
    e = np.ascontiguousarray(np.asarray(g.edges, dtype=np.int32).reshape(-1))
    c, nn = ctypes.c_double(), ctypes.c_double()
    lib().optu_expectation(g.n, g.m, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                           ctypes.c_void_p(np.ascontiguousarray(psi).ctypes.data), ctypes.byref(c), ctypes.byref(nn))
    return c.value, nn.value
