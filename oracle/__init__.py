"""Test infrastructure only: ctypes wrapper of the plain C QAOA oracle (``qaoa_oracle.c``).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg
may import this package.  The CUDA product path never does, and the two share no code.

Every function follows the paper's standard gate-level simulation (Algorithm 1, Section 2.1)
in complex128; the cut value is the plain loop over edges.  Algorithm 3's popcount step is
exposed separately (``alg3_term``/``alg3_cut``) so that the paper's worked example
(Section 2.3, Fig. popcount) can pin it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qaoa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP).  Returns the shared-object path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-Wall", "-Wextra",
               "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        i32p = ctypes.POINTER(ctypes.c_int32)
        dp = ctypes.c_void_p
        L.oracle_cut_value.restype = ctypes.c_double
        L.oracle_cut_value.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, ctypes.c_uint64]
        L.oracle_cut_table.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp]
        L.oracle_alg3_term.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int]
        L.oracle_alg3_cut.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.POINTER(ctypes.c_int)]
        L.oracle_alg2_tot_rotation.restype = ctypes.c_double
        L.oracle_alg2_tot_rotation.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, ctypes.c_uint64]
        L.oracle_initial_layer.argtypes = [ctypes.c_int, dp]
        L.oracle_cost_layer.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, ctypes.c_double, dp]
        L.oracle_mixer_layer.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        L.oracle_qaoa.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, ctypes.c_int, dp, dp, dp]
        L.oracle_expectation.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, dp, dp, dp]
        L.oracle_adjoint_gradient.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp, ctypes.c_int,
                                              dp, dp, dp, dp, dp]
        L.oracle_brute_maxcut.restype = ctypes.c_double
        L.oracle_brute_maxcut.argtypes = [ctypes.c_int, ctypes.c_int, i32p, dp]
        L.oracle_threads.restype = ctypes.c_int
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = L
    return _lib


def _edges(g):
    e = np.ascontiguousarray(np.asarray(g.edges, dtype=np.int32).reshape(-1))
    return e, e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _weights(g):
    if getattr(g, "weights", None) is None:
        return None, None
    w = np.ascontiguousarray(np.asarray(g.weights, dtype=np.float64))
    return w, ctypes.c_void_p(w.ctypes.data)


def _check(rc):
    if rc != 0:
        raise ValueError(f"oracle returned {rc}")


def cut_value(g, z: int) -> float:
    e, ep = _edges(g)
    w, wp = _weights(g)
    return lib().oracle_cut_value(g.n, g.m, ep, wp, z)


def cut_table(g) -> np.ndarray:
    out = np.empty(1 << g.n, dtype=np.uint16)
    e, ep = _edges(g)
    _check(lib().oracle_cut_table(g.n, g.m, ep, ctypes.c_void_p(out.ctypes.data)))
    return out


def alg3_term(b: int, graph_row: int, i: int) -> int:
    return lib().oracle_alg3_term(b, graph_row, i)


def alg3_cut(n: int, graph_I, tot_edge: int, b: int):
    arr = np.ascontiguousarray(np.asarray(graph_I, dtype=np.uint64))
    tr = ctypes.c_int(0)
    c = lib().oracle_alg3_cut(n, ctypes.c_void_p(arr.ctypes.data), tot_edge, b, ctypes.byref(tr))
    return c, tr.value


def alg2_tot_rotation(g, b: int) -> float:
    e, ep = _edges(g)
    w, wp = _weights(g)
    return lib().oracle_alg2_tot_rotation(g.n, g.m, ep, wp, b)


def initial_state(n: int) -> np.ndarray:
    psi = np.empty(1 << n, dtype=np.complex128)
    lib().oracle_initial_layer(n, ctypes.c_void_p(psi.ctypes.data))
    return psi


def cost_layer(g, gamma: float, psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    e, ep = _edges(g)
    w, wp = _weights(g)
    _check(lib().oracle_cost_layer(g.n, g.m, ep, wp, float(gamma), ctypes.c_void_p(psi.ctypes.data)))
    return psi


def mixer_layer(n: int, beta: float, psi: np.ndarray) -> np.ndarray:
    psi = np.ascontiguousarray(psi, dtype=np.complex128).copy()
    lib().oracle_mixer_layer(n, float(beta), ctypes.c_void_p(psi.ctypes.data))
    return psi


def qaoa_state(g, gamma, beta) -> np.ndarray:
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    psi = np.empty(1 << g.n, dtype=np.complex128)
    e, ep = _edges(g)
    w, wp = _weights(g)
    _check(lib().oracle_qaoa(g.n, g.m, ep, wp, len(gamma), ctypes.c_void_p(gamma.ctypes.data),
                             ctypes.c_void_p(beta.ctypes.data), ctypes.c_void_p(psi.ctypes.data)))
    return psi


def expectation(g, psi: np.ndarray):
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    c = ctypes.c_double()
    nn = ctypes.c_double()
    e, ep = _edges(g)
    w, wp = _weights(g)
    _check(lib().oracle_expectation(g.n, g.m, ep, wp, ctypes.c_void_p(psi.ctypes.data),
                                    ctypes.byref(c), ctypes.byref(nn)))
    return c.value, nn.value


def adjoint_gradient(g, gamma, beta):
    gamma = np.ascontiguousarray(gamma, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    p = len(gamma)
    dg = np.zeros(p)
    db = np.zeros(p)
    c = ctypes.c_double()
    e, ep = _edges(g)
    w, wp = _weights(g)
    _check(lib().oracle_adjoint_gradient(g.n, g.m, ep, wp, p, ctypes.c_void_p(gamma.ctypes.data),
                                         ctypes.c_void_p(beta.ctypes.data), ctypes.byref(c),
                                         ctypes.c_void_p(dg.ctypes.data), ctypes.c_void_p(db.ctypes.data)))
    return c.value, dg, db


def brute_maxcut(g) -> float:
    e, ep = _edges(g)
    w, wp = _weights(g)
    return lib().oracle_brute_maxcut(g.n, g.m, ep, wp)


def threads() -> int:
    return lib().oracle_threads()


def set_threads(t: int) -> None:
    lib().oracle_set_threads(t)
