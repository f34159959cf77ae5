"""Thin ctypes binding of ``include/qaoa.h`` (argument marshalling only).

Every function here has the name of the C entry point it calls and does nothing but convert
arguments; all of the simulation runs in ``libqaoa_b300.so``.  Importing this module loads the
library and raises ``ImportError`` if it is missing: there is no CPU fallback.

Device memory and streams come from PyTorch: ``QAOAState`` allocates the state buffer with
``torch.empty(..., device="cuda")`` and passes its ``data_ptr()`` and the current stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# QAOA_LIBRARY may name another build of the same library (the index-checking debug build)
LIB_PATH = os.environ.get("QAOA_LIBRARY") or os.path.join(_HERE, "libqaoa_b300.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -m paper_2312_03019_b300.build` "
        "(there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

QAOA_OK = 0
QAOA_PENDING = 1
QAOA_ERR_INVALID = -1
QAOA_ERR_OOM = -2
QAOA_ERR_CUDA = -3
QAOA_ERR_AGAIN = -4
QAOA_ERR_TIMEOUT = -5
QAOA_ERR_UNSUPPORTED = -6
QAOA_C64 = 0
QAOA_C128 = 1

_STATUS = {0: "OK", 1: "PENDING", -1: "INVALID", -2: "OOM", -3: "CUDA", -4: "AGAIN", -5: "TIMEOUT",
           -6: "UNSUPPORTED"}


class QAOAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"QAOA_ERR_{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Graph(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32),
                ("edges", ctypes.POINTER(ctypes.c_int32)), ("weights", ctypes.POINTER(ctypes.c_double))]


class ProfileStats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("pass_launches", ctypes.c_int64),
                ("pass_ms", ctypes.c_double), ("pass_bytes", ctypes.c_double),
                ("synth_launches", ctypes.c_int64), ("synth_ms", ctypes.c_double),
                ("synth_bytes", ctypes.c_double), ("kind_launches", ctypes.c_int64 * 3),
                ("kind_ms", ctypes.c_double * 3)]


_vp = ctypes.c_void_p
_i32 = ctypes.c_int32
_dp = ctypes.POINTER(ctypes.c_double)


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_sig("qaoa_state_bytes", ctypes.c_size_t, [_i32, ctypes.c_int])
_sig("qaoa_state_init", ctypes.c_int, [ctypes.POINTER(_Graph), ctypes.c_int, _vp, ctypes.c_size_t, _vp,
                                        ctypes.POINTER(_vp)])
_sig("qaoa_state_reset", ctypes.c_int, [_vp])
_sig("qaoa_state_sync", ctypes.c_int, [_vp])
_sig("qaoa_apply_layers", ctypes.c_int, [_vp, _i32, _dp, _dp])
_sig("qaoa_expectation", ctypes.c_int, [_vp, _dp, _dp])
_sig("qaoa_gradient", ctypes.c_int, [_vp, _i32, _dp, _dp, _vp, ctypes.c_size_t, _dp, _dp, _dp])
_sig("qaoa_state_copy_out", ctypes.c_int, [_vp, _vp, ctypes.c_size_t])
_sig("qaoa_state_free", ctypes.c_int, [_vp])
_sig("qaoa_cut_table", ctypes.c_int, [ctypes.POINTER(_Graph), _vp])
_sig("qaoa_cut_table_geometry", ctypes.c_int, [ctypes.POINTER(_Graph), ctypes.c_int, _i32, _i32, _vp])
_sig("qaoa_cut_table_f64", ctypes.c_int, [ctypes.POINTER(_Graph), ctypes.c_int, _i32, _i32, _vp])
_sig("qaoa_plan_describe", ctypes.c_int, [_i32, ctypes.c_int, _i32, ctypes.POINTER(_i32), _i32,
                                           ctypes.POINTER(_i32)])
_sig("qaoa_profile_enable", ctypes.c_int, [_vp, _i32])
_sig("qaoa_profile_read", ctypes.c_int, [_vp, ctypes.POINTER(ProfileStats)])
_sig("qaoa_debug_bounds_read", ctypes.c_int, [_i32, ctypes.POINTER(ctypes.c_uint32), _i32])
_sig("qaoa_expectation_static", ctypes.c_int, [ctypes.POINTER(_Graph), ctypes.c_int, _vp, ctypes.c_size_t, _vp, _dp, _dp])
SERVE_MAX_P = 64


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_inflight", _i32), ("queue_capacity", _i32),
                ("max_batch", _i32), ("streams", _i32), ("use_graphs", _i32), ("prec", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("graph", _Graph), ("p", _i32), ("gamma", _dp), ("beta", _dp), ("want_grad", _i32),
                ("deadline_s", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", _i32), ("p", _i32), ("has_grad", _i32), ("batched", _i32),
                ("expectation", ctypes.c_double), ("norm", ctypes.c_double), ("t_submit", ctypes.c_double),
                ("t_start", ctypes.c_double), ("t_done", ctypes.c_double),
                ("d_gamma", ctypes.c_double * SERVE_MAX_P), ("d_beta", ctypes.c_double * SERVE_MAX_P)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("failed", ctypes.c_int64),
                ("rejected_full", ctypes.c_int64), ("batches", ctypes.c_int64), ("batched_requests", ctypes.c_int64),
                ("single_requests", ctypes.c_int64), ("graph_launches", ctypes.c_int64),
                ("arena_peak_bytes", ctypes.c_size_t), ("timed_out", ctypes.c_int64),
                ("tiled_batches", ctypes.c_int64), ("tiled_batched_requests", ctypes.c_int64)]


_sig("qaoa_server_create", ctypes.c_int, [ctypes.POINTER(ServerConfig), ctypes.POINTER(_vp)])
_sig("qaoa_submit", ctypes.c_int, [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)])
_sig("qaoa_poll", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(Result)])
_sig("qaoa_server_time", ctypes.c_double, [_vp])
_sig("qaoa_server_stats_read", ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)])
_sig("qaoa_server_destroy", ctypes.c_int, [_vp])
_sig("qaoa_last_error", ctypes.c_char_p, [])


def qaoa_last_error() -> str:
    return _lib.qaoa_last_error().decode()


def _check(st: int) -> int:
    if st < 0:
        raise QAOAError(st, qaoa_last_error())
    return st


def _prec(prec) -> int:
    if prec in (QAOA_C64, "c64", "complex64"):
        return QAOA_C64
    if prec in (QAOA_C128, "c128", "complex128"):
        return QAOA_C128
    raise ValueError(f"unknown precision {prec!r}")


def _graph(g):
    """Marshal an object with .n, .edges ([m, 2] ints) and optional .weights."""
    e = np.ascontiguousarray(np.asarray(g.edges, dtype=np.int32).reshape(-1))
    w = getattr(g, "weights", None)
    w = None if w is None else np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    s = _Graph(int(g.n), int(e.size // 2), e.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
               w.ctypes.data_as(_dp) if w is not None else None)
    return s, (e, w)  # keep arrays alive


def qaoa_state_bytes(n: int, prec="c64") -> int:
    return int(_lib.qaoa_state_bytes(int(n), _prec(prec)))


def qaoa_state_init(g, prec, dev_ptr: int, nbytes: int, stream: int = 0) -> int:
    gs, keep = _graph(g)
    h = _vp()
    _check(_lib.qaoa_state_init(ctypes.byref(gs), _prec(prec), _vp(dev_ptr), nbytes, _vp(stream), ctypes.byref(h)))
    return h.value


def qaoa_state_reset(h: int) -> None:
    _check(_lib.qaoa_state_reset(_vp(h)))


def qaoa_state_sync(h: int) -> None:
    _check(_lib.qaoa_state_sync(_vp(h)))


def qaoa_apply_layers(h: int, gamma, beta) -> None:
    ga = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(-1))
    be = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(-1))
    if ga.size != be.size:
        raise ValueError("gamma and beta must have the same length")
    _check(_lib.qaoa_apply_layers(_vp(h), int(ga.size), ga.ctypes.data_as(_dp), be.ctypes.data_as(_dp)))


def qaoa_expectation(h: int):
    c = ctypes.c_double()
    nn = ctypes.c_double()
    _check(_lib.qaoa_expectation(_vp(h), ctypes.byref(c), ctypes.byref(nn)))
    return c.value, nn.value


def qaoa_gradient(h: int, gamma, beta, work_ptr: int, work_bytes: int):
    """(<C>, d<C>/d gamma, d<C>/d beta) by a forward run and an adjoint sweep on the GPU."""
    ga = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(-1))
    be = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(-1))
    if ga.size != be.size:
        raise ValueError("gamma and beta must have the same length")
    dg = np.zeros(ga.size)
    db = np.zeros(ga.size)
    c = ctypes.c_double()
    _check(_lib.qaoa_gradient(_vp(h), int(ga.size), ga.ctypes.data_as(_dp), be.ctypes.data_as(_dp), _vp(work_ptr),
                              work_bytes, ctypes.byref(c), dg.ctypes.data_as(_dp), db.ctypes.data_as(_dp)))
    return c.value, dg, db


def qaoa_expectation_static(g, prec, dev_ptr: int, nbytes: int, stream: int = 0):
    """<C> and norm of a device state without any allocation (scratch is a static device array)."""
    gs, keep = _graph(g)
    c = ctypes.c_double()
    nn = ctypes.c_double()
    _check(_lib.qaoa_expectation_static(ctypes.byref(gs), _prec(prec), _vp(dev_ptr), nbytes, _vp(stream),
                                        ctypes.byref(c), ctypes.byref(nn)))
    return c.value, nn.value


def qaoa_state_copy_out(h: int, n: int, prec) -> np.ndarray:
    dt = np.complex64 if _prec(prec) == QAOA_C64 else np.complex128
    out = np.empty(1 << n, dtype=dt)
    _check(_lib.qaoa_state_copy_out(_vp(h), _vp(out.ctypes.data), out.nbytes))
    return out


def qaoa_state_free(h: int) -> None:
    _check(_lib.qaoa_state_free(_vp(h)))


def qaoa_cut_table(g) -> np.ndarray:
    gs, keep = _graph(g)
    out = np.empty(1 << int(g.n), dtype=np.uint16)
    _check(_lib.qaoa_cut_table(ctypes.byref(gs), _vp(out.ctypes.data)))
    return out


def qaoa_cut_table_f64(g, prec="c64", group: int = -1, layout: int = 0) -> np.ndarray:
    """C(z) for every z as doubles (unit or edge-weighted graphs), from the device evaluation."""
    gs, keep = _graph(g)
    out = np.empty(1 << int(g.n), dtype=np.float64)
    _check(_lib.qaoa_cut_table_f64(ctypes.byref(gs), _prec(prec), int(group), int(layout), _vp(out.ctypes.data)))
    return out


def qaoa_cut_table_geometry(g, prec, group: int, layout: int) -> np.ndarray:
    gs, keep = _graph(g)
    out = np.empty(1 << int(g.n), dtype=np.uint16)
    _check(_lib.qaoa_cut_table_geometry(ctypes.byref(gs), _prec(prec), int(group), int(layout),
                                        _vp(out.ctypes.data)))
    return out


def qaoa_plan_describe(n: int, prec, p: int) -> list:
    cnt = _i32()
    _check(_lib.qaoa_plan_describe(int(n), _prec(prec), int(p), None, 0, ctypes.byref(cnt)))
    buf = (_i32 * max(1, cnt.value))()
    _check(_lib.qaoa_plan_describe(int(n), _prec(prec), int(p), buf, cnt.value, ctypes.byref(cnt)))
    return list(buf[: cnt.value])


def qaoa_debug_bounds_read(device: int = 0, clear: bool = True) -> int:
    """The index-check word of a debug build (0: no check failed); raises QAOAError with
    QAOA_ERR_UNSUPPORTED on a release build."""
    f = ctypes.c_uint32()
    _check(_lib.qaoa_debug_bounds_read(int(device), ctypes.byref(f), 1 if clear else 0))
    return f.value


def qaoa_profile_enable(h: int, enable: bool = True) -> None:
    _check(_lib.qaoa_profile_enable(_vp(h), 1 if enable else 0))


def qaoa_profile_read(h: int) -> dict:
    st = ProfileStats()
    _check(_lib.qaoa_profile_read(_vp(h), ctypes.byref(st)))
    out = {k: getattr(st, k) for k, _ in ProfileStats._fields_}
    out["kind_launches"] = list(st.kind_launches)
    out["kind_ms"] = list(st.kind_ms)
    return out


class QAOAState:
    """A state of ``g.n`` qubits in a torch-allocated device buffer, bound to the current stream."""

    def __init__(self, g, prec="c64", device=None, stream=None):
        import torch

        self.n = int(g.n)
        self.prec = _prec(prec)
        self.nbytes = qaoa_state_bytes(self.n, self.prec)
        if self.nbytes == 0:
            raise ValueError("n out of range")
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.buffer = torch.empty(self.nbytes, dtype=torch.uint8, device=dev)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        with torch.cuda.device(dev):
            self.handle = qaoa_state_init(g, self.prec, self.buffer.data_ptr(), self.nbytes,
                                          self.stream.cuda_stream)

    def reset(self):
        qaoa_state_reset(self.handle)
        return self

    def apply_layers(self, gamma, beta):
        qaoa_apply_layers(self.handle, gamma, beta)
        return self

    def expectation(self):
        return qaoa_expectation(self.handle)

    def gradient(self, gamma, beta):
        """(<C>, d<C>/d gamma, d<C>/d beta) after len(gamma) levels from |+>^n by the adjoint sweep
        (qaoa_gradient); the sweep's second state lives in a work buffer kept with this handle.
        The state is |+>^n again afterwards."""
        import torch

        if getattr(self, "_work", None) is None:
            self._work = torch.empty(self.nbytes, dtype=torch.uint8, device=self.buffer.device)
        return qaoa_gradient(self.handle, gamma, beta, self._work.data_ptr(), self.nbytes)

    def amplitudes(self) -> np.ndarray:
        return qaoa_state_copy_out(self.handle, self.n, self.prec)

    def as_tensor(self):
        """The device buffer viewed as a complex torch tensor, index z = amplitude of z."""
        import torch

        qaoa_state_sync(self.handle)

        dt = torch.complex64 if self.prec == QAOA_C64 else torch.complex128
        return self.buffer.view(dt)

    def close(self):
        if getattr(self, "handle", None):
            qaoa_state_free(self.handle)
            self.handle = None
        self.buffer = None
        self._work = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qaoa_server_create(hbm_budget_bytes: int, prec="c64", max_inflight: int = 64, queue_capacity: int = 8192,
                       max_batch: int = 64, streams: int = 8, use_graphs: bool = True) -> int:
    cfg = ServerConfig(int(hbm_budget_bytes), int(max_inflight), int(queue_capacity), int(max_batch), int(streams),
                       1 if use_graphs else 0, _prec(prec))
    h = _vp()
    _check(_lib.qaoa_server_create(ctypes.byref(cfg), ctypes.byref(h)))
    return h.value


def qaoa_submit(sv: int, g, gamma, beta, want_grad: bool = False, deadline_s: float = 0.0) -> int:
    """Returns the ticket; raises QAOAError (status QAOA_ERR_AGAIN when the queue is full).
    deadline_s > 0: a request not dispatched within that many seconds completes with status
    QAOA_ERR_TIMEOUT without running."""
    gs, keep = _graph(g)
    ga = np.ascontiguousarray(np.asarray(gamma, dtype=np.float64).reshape(-1))
    be = np.ascontiguousarray(np.asarray(beta, dtype=np.float64).reshape(-1))
    req = Request(gs, int(ga.size), ga.ctypes.data_as(_dp), be.ctypes.data_as(_dp), 1 if want_grad else 0,
                  float(deadline_s))
    t = ctypes.c_uint64()
    _check(_lib.qaoa_submit(_vp(sv), ctypes.byref(req), ctypes.byref(t)))
    return t.value


def qaoa_poll(sv: int, ticket: int):
    """None while pending, else a dict with the result (the ticket is released)."""
    r = Result()
    st = _check(_lib.qaoa_poll(_vp(sv), ctypes.c_uint64(ticket), ctypes.byref(r)))
    if st == QAOA_PENDING:
        return None
    out = {k: getattr(r, k) for k, _ in Result._fields_ if k not in ("d_gamma", "d_beta")}
    out["d_gamma"] = np.array(r.d_gamma[: r.p]) if r.has_grad else None
    out["d_beta"] = np.array(r.d_beta[: r.p]) if r.has_grad else None
    return out


def qaoa_server_time(sv: int) -> float:
    return float(_lib.qaoa_server_time(_vp(sv)))


def qaoa_server_stats_read(sv: int) -> dict:
    st = ServerStats()
    _check(_lib.qaoa_server_stats_read(_vp(sv), ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


def qaoa_server_destroy(sv: int) -> None:
    _check(_lib.qaoa_server_destroy(_vp(sv)))
