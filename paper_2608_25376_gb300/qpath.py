"""Thin ctypes binding of libqpath (include/qpath.h), names as in the C ABI.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Buffers may be torch tensors (host or CUDA) or numpy arrays; they are
passed by pointer and owned by the caller.  The library must be built
(``paper_2608_25376_gb300.build.build()``); loading fails loudly if it is not.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

QP_OK, QP_EINVAL, QP_ENOMEM, QP_ERANGE, QP_ECUDA, QP_ETIMEOUT, QP_EINFEASIBLE = range(7)
QP_DENSE, QP_STRUCTURED, QP_DIST_I16 = 1, 2, 4
QP_KERNEL_AUTO, QP_KERNEL_DENSE, QP_KERNEL_STRUCTURED, QP_KERNEL_STRUCTURED_FLAT = 0, 1, 2, 3
QP_KERNEL_STRUCTURED_ROWS, QP_KERNEL_STRUCTURED_GROUP, QP_KERNEL_STRUCTURED_ROWS_SHARED = 4, 5, 6
QP_ANNEAL_SKIP_SETTLED = 1
QP_BATCH_D_SHARED = 2
E_NONE = np.iinfo(np.int64).max

# every entry point include/qpath.h declares
SYMBOLS = ["qp_build_qubo", "qp_build_qubo_weighted", "qp_build_from_dense", "qp_qubo_info", "qp_export_dense", "qp_export_dist",
           "qp_thresholds", "qp_anneal", "qp_anneal_ex", "qp_anneal_noalloc", "qp_batch_create",
           "qp_batch_run", "qp_batch_info", "qp_batch_destroy", "qp_anneal_batch", "qp_decode_path",
           "qp_decode_batch", "qp_repair_batch", "qp_repair_path", "qp_anneal_timed", "qp_anneal_pt", "qp_ws_create", "qp_ws_destroy", "qp_ws_param_count", "qp_ws_get_params",
           "qp_ws_set_params", "qp_ws_features", "qp_ws_forward", "qp_ws_set_forward_mode", "qp_ws_grads", "qp_ws_train_step",
           "qp_ws_get_state", "qp_ws_get_buffer", "qp_ws_expected_steps", "qp_ws_walk", "qp_ws_greedy",
           "qp_ws_decode", "qp_ws_decode_walk", "qp_ws_infer", "qp_selftest_wait", "qp_device_checks", "qp_destroy",
           "qp_last_error"]


class QpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qpath status {status}: {msg}")
        self.status = status


class qp_field(ct.Structure):
    _fields_ = [("rows", ct.c_int32), ("cols", ct.c_int32), ("free_mask", ct.c_void_p), ("start", ct.c_int32)]


class qp_schedule(ct.Structure):
    _fields_ = [("n_sweeps", ct.c_int32), ("T0", ct.c_double), ("T1", ct.c_double),
                ("sweep_begin", ct.c_int32), ("sweep_end", ct.c_int32)]


class qp_batch_opts(ct.Structure):
    _fields_ = [("replicas_per_cta", ct.c_int32), ("ctas", ct.c_int32), ("flags", ct.c_int32)]


class qp_timed_info(ct.Structure):
    _fields_ = [("n_sweeps", ct.c_int32), ("rounds", ct.c_int32), ("replica", ct.c_int32), ("status", ct.c_int32),
                ("n_feasible", ct.c_int64), ("energy", ct.c_int64), ("probe_ms", ct.c_double),
                ("elapsed_ms", ct.c_double)]


class qp_pt_schedule(ct.Structure):
    _fields_ = [("levels", ct.c_int32), ("T_lo", ct.c_double), ("T_hi", ct.c_double),
                ("sweeps_per_exchange", ct.c_int32), ("exchanges", ct.c_int32)]


def pt_schedule(levels, T_lo, T_hi, sweeps_per_exchange, exchanges) -> qp_pt_schedule:
    return qp_pt_schedule(int(levels), float(T_lo), float(T_hi), int(sweeps_per_exchange), int(exchanges))


class qp_anneal_opts(ct.Structure):
    _fields_ = [("kernel", ct.c_int32), ("replicas_per_cta", ct.c_int32), ("replica_offset", ct.c_int32),
                ("accepts_out", ct.c_void_p), ("flags", ct.c_int32)]


def lib_path() -> str:
    """The library to load: QPATH_LIBRARY when set (e.g. the checked build), else the release build."""
    return os.environ.get("QPATH_LIBRARY") or _build.LIB


def lib():
    """Load libqpath.so (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = lib_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libqpath is not built ({path} missing): run __graft_entry__.build()")
            L = ct.CDLL(path)
            vp, i32, i64, u64 = ct.c_void_p, ct.c_int32, ct.c_int64, ct.c_uint64
            P = ct.POINTER
            sig = {
                "qp_build_qubo": [P(qp_field), i32, i32, i32, i32, P(vp)],
                "qp_build_qubo_weighted": [P(qp_field), i32, vp, i32, i32, P(vp)],
                "qp_build_from_dense": [vp, i64, vp, vp, i64, P(vp)],
                "qp_qubo_info": [vp, P(i64), P(i32), P(i64), P(i32), P(i32)],
                "qp_export_dense": [vp, vp],
                "qp_export_dist": [vp, vp],
                "qp_thresholds": [P(qp_schedule), i32, vp, i32, P(i32)],
                "qp_anneal": [vp, i32, P(qp_schedule), u64, vp, vp, vp, vp, vp],
                "qp_anneal_ex": [vp, i32, P(qp_schedule), u64, vp, vp, vp, vp, P(qp_anneal_opts), vp],
                "qp_anneal_noalloc": [vp, i32, P(qp_schedule), u64, vp, vp, vp, vp, i32, vp],
                "qp_batch_create": [P(vp), i32, i32, P(qp_schedule), u64, P(vp), P(vp), P(vp),
                                    P(qp_batch_opts), P(vp)],
                "qp_batch_run": [vp, vp],
                "qp_batch_info": [vp, P(i32), P(i32), P(i32)],
                "qp_anneal_batch": [P(vp), i32, i32, P(qp_schedule), u64, P(vp), P(vp), P(vp), vp],
                "qp_ws_create": [u64, P(vp)],
                "qp_ws_get_params": [vp, vp],
                "qp_ws_set_params": [vp, vp],
                "qp_ws_features": [P(qp_field), vp, P(i32)],
                "qp_ws_forward": [vp, vp, i32, vp, vp],
                "qp_ws_set_forward_mode": [vp, i32],
                "qp_ws_grads": [vp, vp, vp, vp, i32, vp, vp, vp],
                "qp_ws_train_step": [vp, vp, vp, vp, i32, ct.c_float, vp, vp],
                "qp_ws_get_state": [vp, i32, vp],
                "qp_ws_expected_steps": [vp, i32, i32, vp, vp, vp],
                "qp_ws_walk": [vp, vp, i32, vp, vp, vp, vp],
                "qp_ws_greedy": [vp, i32, i32, i32, vp, vp, vp],
                "qp_ws_get_buffer": [vp, i32, i32, vp],
                "qp_ws_decode": [vp, i32, i32, i32, vp, vp],
                "qp_ws_decode_walk": [vp, i32, i32, i32, vp, vp, vp],
                "qp_ws_infer": [vp, P(qp_field), vp, vp, vp, vp],
                "qp_selftest_wait": [P(i32), P(ct.c_double)],
                "qp_device_checks": [P(i32), P(ct.c_uint32)],
                "qp_decode_path": [vp, vp, vp, vp],
                "qp_decode_batch": [vp, i32, vp, vp, vp, vp],
                "qp_repair_batch": [vp, i32, vp, i32, vp, vp, vp, vp],
                "qp_repair_path": [vp, vp, i32, vp, P(i64), P(i32)],
                "qp_anneal_pt": [vp, i32, P(qp_pt_schedule), u64, vp, vp, vp, vp, vp, vp, vp],
                "qp_anneal_timed": [vp, i32, P(qp_schedule), u64, ct.c_double, i32, vp, P(i64), vp,
                                    P(qp_timed_info), vp],
            }
            for name, args in sig.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = ct.c_int
            L.qp_ws_destroy.argtypes = [vp]
            L.qp_ws_destroy.restype = None
            L.qp_ws_param_count.argtypes = []
            L.qp_ws_param_count.restype = i64
            L.qp_batch_destroy.argtypes = [vp]
            L.qp_batch_destroy.restype = None
            L.qp_destroy.argtypes = [vp]
            L.qp_destroy.restype = None
            L.qp_last_error.argtypes = []
            L.qp_last_error.restype = ct.c_char_p
            _lib = L
    return _lib


def qp_last_error() -> str:
    return lib().qp_last_error().decode()


def _check(status):
    if status != QP_OK:
        raise QpError(status, qp_last_error())


def _ptr(x):
    """Address of a torch tensor / numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("buffers must be contiguous")
        return ct.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("buffers must be contiguous")
        return ct.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported buffer type {type(x)}")


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ct.c_void_p(stream.cuda_stream)
    return ct.c_void_p(int(stream))


def schedule(n_sweeps, T0=1e3, T1=1.0, sweep_begin=0, sweep_end=None) -> qp_schedule:
    return qp_schedule(int(n_sweeps), float(T0), float(T1), int(sweep_begin),
                       int(n_sweeps if sweep_end is None else sweep_end))


class Handle:
    """Owns a qp_handle*; freed by qp_destroy on close / garbage collection."""

    def __init__(self, ptr):
        self.ptr = ptr

    def close(self):
        if self.ptr:
            lib().qp_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return qp_qubo_info(self)


def qp_build_qubo(field, A=0, B=1, scale=100, flags=QP_STRUCTURED) -> Handle:
    """field: an object with rows, cols, free_mask (uint8 numpy or None), start."""
    mask = None if field.free_mask is None else np.ascontiguousarray(field.free_mask, np.uint8)
    f = qp_field(int(field.rows), int(field.cols), None if mask is None else mask.ctypes.data, int(field.start))
    out = ct.c_void_p()
    _check(lib().qp_build_qubo(ct.byref(f), int(A), int(B), int(scale), int(flags), ct.byref(out)))
    return Handle(out)


def qp_build_qubo_weighted(field, leg_weights, A=0, scale=100) -> Handle:
    """The path QUBO with one weight per leg on the distance term (C - 1
    non-negative integers; see objectives.payload_leg_weights); the handle
    anneals with the dense kernel."""
    mask = None if field.free_mask is None else np.ascontiguousarray(field.free_mask, np.uint8)
    f = qp_field(int(field.rows), int(field.cols), None if mask is None else mask.ctypes.data, int(field.start))
    w = np.ascontiguousarray(leg_weights, np.int32)
    out = ct.c_void_p()
    _check(lib().qp_build_qubo_weighted(ct.byref(f), int(A), _ptr(w), int(w.size), int(scale), ct.byref(out)))
    return Handle(out)


def qp_build_from_dense(S, c0=0, frozen=None, frozen_val=None) -> Handle:
    S = np.ascontiguousarray(S, np.int32)
    fr = None if frozen is None else np.ascontiguousarray(frozen, np.uint8)
    fv = None if frozen_val is None else np.ascontiguousarray(frozen_val, np.uint8)
    out = ct.c_void_p()
    _check(lib().qp_build_from_dense(_ptr(S), S.shape[0], _ptr(fr), _ptr(fv), int(c0), ct.byref(out)))
    return Handle(out)


def qp_qubo_info(h: Handle) -> dict:
    n, C, c0, md, A = ct.c_int64(), ct.c_int32(), ct.c_int64(), ct.c_int32(), ct.c_int32()
    _check(lib().qp_qubo_info(h.ptr, ct.byref(n), ct.byref(C), ct.byref(c0), ct.byref(md), ct.byref(A)))
    return dict(n=n.value, C=C.value, c0=c0.value, max_d=md.value, A=A.value)


def qp_export_dense(h: Handle) -> np.ndarray:
    n = qp_qubo_info(h)["n"]
    S = np.zeros((n, n), np.int32)
    _check(lib().qp_export_dense(h.ptr, _ptr(S)))
    return S


def qp_export_dist(h: Handle) -> np.ndarray:
    C = qp_qubo_info(h)["C"]
    d = np.zeros((C, C), np.int32)
    _check(lib().qp_export_dist(h.ptr, _ptr(d)))
    return d


def qp_thresholds(sched: qp_schedule, sweep: int) -> np.ndarray:
    n = ct.c_int32()
    _check(lib().qp_thresholds(ct.byref(sched), int(sweep), None, 0, ct.byref(n)))
    out = np.zeros(n.value, np.uint32)
    _check(lib().qp_thresholds(ct.byref(sched), int(sweep), _ptr(out), n.value, ct.byref(n)))
    return out


def qp_anneal(h: Handle, replicas, sched, seed, init_states, states_out, energies_out, best_out=None,
              stream=None):
    _check(lib().qp_anneal(h.ptr, int(replicas), ct.byref(sched), ct.c_uint64(seed), _ptr(init_states),
                           _ptr(states_out), _ptr(energies_out), _ptr(best_out), _stream(stream)))


def qp_anneal_ex(h: Handle, replicas, sched, seed, init_states, states_out, energies_out, best_out=None,
                 kernel=QP_KERNEL_AUTO, replicas_per_cta=0, replica_offset=0, accepts_out=None, stream=None,
                 flags=0):
    o = qp_anneal_opts(int(kernel), int(replicas_per_cta), int(replica_offset),
                       None if accepts_out is None else _ptr(accepts_out).value, int(flags))
    _check(lib().qp_anneal_ex(h.ptr, int(replicas), ct.byref(sched), ct.c_uint64(seed), _ptr(init_states),
                              _ptr(states_out), _ptr(energies_out), _ptr(best_out), ct.byref(o),
                              _stream(stream)))


def qp_anneal_noalloc(h: Handle, replicas, sched, seed, init_states, states_out, energies_out, best_out=None,
                      replica_offset=0, stream=None):
    """The allocation-free structured anneal (device buffers only)."""
    _check(lib().qp_anneal_noalloc(h.ptr, int(replicas), ct.byref(sched), ct.c_uint64(seed), _ptr(init_states),
                                   _ptr(states_out), _ptr(energies_out), _ptr(best_out), int(replica_offset),
                                   _stream(stream)))


def _ptr_array(xs):
    arr = (ct.c_void_p * len(xs))()
    for i, x in enumerate(xs):
        p = _ptr(x)
        arr[i] = None if p is None else p.value
    return arr


class Batch:
    """Owns a qp_batch* (a captured CUDA graph over many fields)."""

    def __init__(self, ptr, keep):
        self.ptr = ptr
        self._keep = keep  # handles and buffers must outlive the batch

    def run(self, stream=None):
        qp_batch_run(self, stream)

    @property
    def info(self):
        return qp_batch_info(self)

    def close(self):
        if self.ptr:
            lib().qp_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qp_batch_create(handles, replicas, sched, seed, states_out, energies_out, best_out=None,
                    replicas_per_cta=0, ctas=0, flags=0) -> Batch:
    hs = (ct.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    so, eo = _ptr_array(states_out), _ptr_array(energies_out)
    bo = None if best_out is None else _ptr_array(best_out)
    o = qp_batch_opts(int(replicas_per_cta), int(ctas), int(flags))
    out = ct.c_void_p()
    _check(lib().qp_batch_create(hs, len(handles), int(replicas), ct.byref(sched), ct.c_uint64(seed), so, eo,
                                 bo, ct.byref(o), ct.byref(out)))
    return Batch(out, (handles, states_out, energies_out, best_out))


def qp_batch_run(b: Batch, stream=None):
    _check(lib().qp_batch_run(b.ptr, _stream(stream)))


def qp_batch_info(b: Batch) -> dict:
    w, c, u = ct.c_int32(), ct.c_int32(), ct.c_int32()
    _check(lib().qp_batch_info(b.ptr, ct.byref(w), ct.byref(c), ct.byref(u)))
    return dict(replicas_per_cta=w.value, ctas=c.value, units=u.value)


def qp_batch_destroy(b: Batch):
    b.close()


def qp_anneal_batch(handles, replicas, sched, seed, states_out, energies_out, best_out=None, stream=None):
    hs = (ct.c_void_p * len(handles))(*[h.ptr.value for h in handles])
    so, eo = _ptr_array(states_out), _ptr_array(energies_out)
    bo = None if best_out is None else _ptr_array(best_out)
    _check(lib().qp_anneal_batch(hs, len(handles), int(replicas), ct.byref(sched), ct.c_uint64(seed), so, eo, bo,
                                 _stream(stream)))


def qp_decode_path(h: Handle, state):
    """-> (path int32[C], length) or None when the state is not a path."""
    C = qp_qubo_info(h)["C"]
    path = np.zeros(C, np.int32)
    L = ct.c_int64()
    st = lib().qp_decode_path(h.ptr, _ptr(state), _ptr(path), ct.byref(L))
    if st == QP_EINFEASIBLE:
        return None
    _check(st)
    return path, L.value


def qp_decode_batch(h: Handle, replicas, states, paths_out, lengths_out, stream=None):
    _check(lib().qp_decode_batch(h.ptr, int(replicas), _ptr(states), _ptr(paths_out), _ptr(lengths_out),
                                 _stream(stream)))


def qp_anneal_pt(h: Handle, groups, pt, seed, init_states, states_out, energies_out, best_out=None,
                 levels_out=None, swaps_out=None, stream=None):
    _check(lib().qp_anneal_pt(h.ptr, int(groups), ct.byref(pt), ct.c_uint64(seed), _ptr(init_states),
                              _ptr(states_out), _ptr(energies_out), _ptr(best_out), _ptr(levels_out),
                              _ptr(swaps_out), _stream(stream)))


REPAIR_KEPT, REPAIR_SHORTENED, REPAIR_FIXED = 0, 1, 2


def qp_repair_batch(h: Handle, replicas, states, max_passes, paths_out, lengths_out, status_out=None,
                    stream=None):
    _check(lib().qp_repair_batch(h.ptr, int(replicas), _ptr(states), int(max_passes), _ptr(paths_out),
                                 _ptr(lengths_out), _ptr(status_out), _stream(stream)))


def qp_repair_path(h: Handle, state, max_passes=0):
    """-> (path int32[C], length, status)"""
    C = qp_qubo_info(h)["C"]
    path = np.zeros(C, np.int32)
    L, S = ct.c_int64(), ct.c_int32()
    _check(lib().qp_repair_path(h.ptr, _ptr(state), int(max_passes), _ptr(path), ct.byref(L), ct.byref(S)))
    return path, L.value, S.value


def qp_anneal_timed(h: Handle, replicas, sched, seed, time_limit_ms, max_passes=0, want_state=False,
                    stream=None) -> dict:
    """-> {"path", "length", "state" (or None), and every qp_timed_info field}"""
    info = qp_qubo_info(h)
    path = np.zeros(info["C"], np.int32)
    state = np.zeros(info["n"], np.uint8) if want_state else None
    L = ct.c_int64()
    ti = qp_timed_info()
    _check(lib().qp_anneal_timed(h.ptr, int(replicas), ct.byref(sched), ct.c_uint64(seed), float(time_limit_ms),
                                 int(max_passes), _ptr(path), ct.byref(L), _ptr(state), ct.byref(ti),
                                 _stream(stream)))
    out = {"path": path, "length": L.value, "state": state}
    out.update({k: getattr(ti, k) for k, _ in qp_timed_info._fields_})
    return out


def qp_destroy(h: Handle):
    h.close()


# --------------------------------------------------------------------------- learned warm start
WS_FEATURES, WS_STEPS = 16, 256
QP_WS_FORWARD_FUSED, QP_WS_FORWARD_LAYERED = 0, 1


class WarmStartModel:
    """Owns a qp_ws* (the per-cell step-logit MLP)."""

    def __init__(self, seed=0):
        out = ct.c_void_p()
        _check(lib().qp_ws_create(ct.c_uint64(seed), ct.byref(out)))
        self.ptr = out

    def close(self):
        if self.ptr:
            lib().qp_ws_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qp_ws_param_count() -> int:
    return int(lib().qp_ws_param_count())


def qp_ws_get_params(m: WarmStartModel) -> np.ndarray:
    out = np.zeros(qp_ws_param_count(), np.float32)
    _check(lib().qp_ws_get_params(m.ptr, _ptr(out)))
    return out


def qp_ws_set_params(m: WarmStartModel, params):
    p = np.ascontiguousarray(params, np.float32)
    assert p.size == qp_ws_param_count()
    _check(lib().qp_ws_set_params(m.ptr, _ptr(p)))


def qp_ws_features(field) -> np.ndarray:
    mask = None if field.free_mask is None else np.ascontiguousarray(field.free_mask, np.uint8)
    f = qp_field(int(field.rows), int(field.cols), None if mask is None else mask.ctypes.data, int(field.start))
    C = ct.c_int32()
    _check(lib().qp_ws_features(ct.byref(f), None, ct.byref(C)))
    out = np.zeros((C.value, WS_FEATURES), np.float32)
    _check(lib().qp_ws_features(ct.byref(f), _ptr(out), ct.byref(C)))
    return out


def qp_ws_forward(m: WarmStartModel, feats, logits_out=None, stream=None):
    x = np.ascontiguousarray(feats, np.float32)
    M = x.shape[0]
    out = np.zeros((M, WS_STEPS), np.float32) if logits_out is None else logits_out
    _check(lib().qp_ws_forward(m.ptr, _ptr(x), M, _ptr(out), _stream(stream)))
    return out


def qp_ws_set_forward_mode(m: WarmStartModel, mode: int):
    _check(lib().qp_ws_set_forward_mode(m.ptr, int(mode)))


def qp_ws_grads(m: WarmStartModel, feats, labels, steps, stream=None):
    x = np.ascontiguousarray(feats, np.float32)
    lb = np.ascontiguousarray(labels, np.int32)
    sp = np.ascontiguousarray(steps, np.int32)
    g = np.zeros(qp_ws_param_count(), np.float32)
    loss = ct.c_float()
    _check(lib().qp_ws_grads(m.ptr, _ptr(x), _ptr(lb), _ptr(sp), x.shape[0], _ptr(g), ct.byref(loss),
                             _stream(stream)))
    return loss.value, g


def qp_ws_train_step(m: WarmStartModel, feats, labels, steps, lr, stream=None) -> float:
    x = np.ascontiguousarray(feats, np.float32)
    lb = np.ascontiguousarray(labels, np.int32)
    sp = np.ascontiguousarray(steps, np.int32)
    loss = ct.c_float()
    _check(lib().qp_ws_train_step(m.ptr, _ptr(x), _ptr(lb), _ptr(sp), x.shape[0], ct.c_float(lr), ct.byref(loss),
                                  _stream(stream)))
    return loss.value


QP_WS_STATE_PARAMS, QP_WS_STATE_ADAM_M, QP_WS_STATE_ADAM_V, QP_WS_STATE_GRADS = 0, 1, 2, 3
QP_WS_BUF_X0, QP_WS_BUF_H1, QP_WS_BUF_H2, QP_WS_BUF_H3, QP_WS_BUF_Z, QP_WS_BUF_DZ = 0, 1, 2, 3, 4, 5
QP_WS_BUF_DH1, QP_WS_BUF_DH2, QP_WS_BUF_DH3, QP_WS_BUF_W_BF16, QP_WS_BUF_WT_BF16 = 6, 7, 8, 16, 32


def qp_ws_get_state(m: WarmStartModel, which: int) -> np.ndarray:
    """fp32 master parameters, Adam moments or last gradients (flat get/set layout)."""
    out = np.zeros(qp_ws_param_count(), np.float32)
    _check(lib().qp_ws_get_state(m.ptr, int(which), _ptr(out)))
    return out


def qp_ws_get_buffer(m: WarmStartModel, which: int, rows: int = 0) -> np.ndarray:
    """Rows of an activation / gradient buffer of the last pass (bf16 buffers as
    uint16 bits, Z as float32), or a layer's bf16 weight copy (uint16 bits)."""
    dims = [(256, 16), (256, 256), (256, 256), (256, 256)]
    if which >= QP_WS_BUF_WT_BF16:
        no, ni = dims[which - QP_WS_BUF_WT_BF16]
        out = np.zeros((ni, no), np.uint16)
    elif which >= QP_WS_BUF_W_BF16:
        no, ni = dims[which - QP_WS_BUF_W_BF16]
        out = np.zeros((no, ni), np.uint16)
    elif which == QP_WS_BUF_Z:
        out = np.zeros((rows, WS_STEPS), np.float32)
    else:
        out = np.zeros((rows, WS_FEATURES if which == QP_WS_BUF_X0 else 256), np.uint16)
    _check(lib().qp_ws_get_buffer(m.ptr, int(which), int(rows), _ptr(out)))
    return out


def bf16_bits_to_float(u) -> np.ndarray:
    """uint16 bfloat16 bit patterns -> float64 values."""
    u = np.asarray(u, np.uint16).astype(np.uint32) << 16
    return u.view(np.float32).astype(np.float64)


def qp_ws_decode(logits, C, start_cell):
    """-> (state uint8 [C*C], path int32 [C])"""
    L = np.ascontiguousarray(logits, np.float32)
    st = np.zeros(C * C, np.uint8)
    path = np.zeros(C, np.int32)
    _check(lib().qp_ws_decode(_ptr(L), L.shape[1], int(C), int(start_cell), _ptr(st), _ptr(path)))
    return st, path


def qp_ws_decode_walk(logits, C, start_cell, d):
    """-> (state uint8 [C*C], path int32 [C]) by the guided nearest-cell walk"""
    L = np.ascontiguousarray(logits, np.float32)
    dd = np.ascontiguousarray(d, np.int32)
    st = np.zeros(C * C, np.uint8)
    path = np.zeros(C, np.int32)
    _check(lib().qp_ws_decode_walk(_ptr(L), L.shape[1], int(C), int(start_cell), _ptr(dd), _ptr(st), _ptr(path)))
    return st, path


def qp_ws_infer(m: WarmStartModel, field, d=None, stream=None):
    """-> (state uint8 [C*C], path int32 [C]): features, logits and the decoded
    seed of one field in one call (guided walk when d is given, else greedy
    matching)."""
    mask = None if field.free_mask is None else np.ascontiguousarray(field.free_mask, np.uint8)
    f = qp_field(int(field.rows), int(field.cols), None if mask is None else mask.ctypes.data, int(field.start))
    C = int(mask.sum()) if mask is not None else field.rows * field.cols
    st = np.zeros(C * C, np.uint8)
    path = np.zeros(C, np.int32)
    dd = None if d is None else np.ascontiguousarray(d, np.int32)
    _check(lib().qp_ws_infer(m.ptr, ct.byref(f), _ptr(dd), _ptr(st), _ptr(path), _stream(stream)))
    return st, path


def qp_ws_expected_steps(logits, steps, E_out=None, stream=None):
    """Expected step per row of device logits [M, ld] over the first steps[m]
    entries (device int32 [M]); -> E (device float32 [M])."""
    import torch
    M, ld = logits.shape
    E = torch.empty(M, dtype=torch.float32, device=logits.device) if E_out is None else E_out
    _check(lib().qp_ws_expected_steps(_ptr(logits), int(ld), int(M), _ptr(steps), _ptr(E), _stream(stream)))
    return E


def qp_ws_walk(h: Handle, score=None, slack=0, state_out=None, path_out=None, length_out=None, stream=None):
    """The walk decode on the device: -> (state uint8 [C*C], path int32 [C],
    length int64 [1]), device tensors (allocated when not given)."""
    import torch
    C = h.info["C"]
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.empty(C * C, dtype=torch.uint8, device=dev) if state_out is None else state_out
    pa = torch.empty(C, dtype=torch.int32, device=dev) if path_out is None else path_out
    ln = torch.empty(1, dtype=torch.int64, device=dev) if length_out is None else length_out
    _check(lib().qp_ws_walk(h.ptr, _ptr(score), int(slack), _ptr(st), _ptr(pa), _ptr(ln), _stream(stream)))
    return st, pa, ln


def qp_ws_greedy(logits, C, start_cell, state_out=None, path_out=None, stream=None):
    """The greedy matching decode (qp_ws_decode) on the device: logits a device
    float32 tensor [C', ld] with C' >= C rows; -> (state uint8 [C*C], path int32
    [C]), device tensors (allocated when not given)."""
    import torch
    ld = logits.shape[1]
    st = torch.empty(C * C, dtype=torch.uint8, device=logits.device) if state_out is None else state_out
    pa = torch.empty(C, dtype=torch.int32, device=logits.device) if path_out is None else path_out
    _check(lib().qp_ws_greedy(_ptr(logits), int(ld), int(C), int(start_cell), _ptr(st), _ptr(pa), _stream(stream)))
    return st, pa


def qp_selftest_wait() -> dict:
    """-> {"timed_out": 1 if the never-completed wait gave up, "waited_ms": ...}"""
    t, w = ct.c_int32(), ct.c_double()
    _check(lib().qp_selftest_wait(ct.byref(t), ct.byref(w)))
    return {"timed_out": t.value, "waited_ms": w.value}


def qp_device_checks():
    """(enabled, first_failure) of the loaded library's device bounds checks; clears the record."""
    en, w = ct.c_int32(), ct.c_uint32()
    _check(lib().qp_device_checks(ct.byref(en), ct.byref(w)))
    return bool(en.value), int(w.value)
