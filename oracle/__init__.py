"""CPU oracle for the one-hot UAV path QUBO annealer -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``qp_oracle.c`` (plain C, one
thread per replica) with ctypes and numpy.  It shares no code with the CUDA
library: the C file restates every step from the paper (Sections II-III,
Eqs. 1-6, Algorithm 1); the readings it takes where the paper is silent are
listed at the top of that file.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

E_NONE = np.iinfo(np.int64).max


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
               "-ffp-contract=off", _SRC, "-o", _LIB + ".tmp", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _p(a, t):
    return a.ctypes.data_as(ct.POINTER(t)) if a is not None else None


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ct.CDLL(_LIB)
            i32, i64, u64, dbl = ct.c_int32, ct.c_int64, ct.c_uint64, ct.c_double
            P = ct.POINTER
            L.or_cells.restype = i32
            L.or_cells.argtypes = [i32, i32, P(ct.c_uint8), i32, P(i32), P(i32), P(i32)]
            L.or_round_scaled_sqrt.restype = i64
            L.or_round_scaled_sqrt.argtypes = [i64, i64]
            L.or_distances.restype = None
            L.or_distances.argtypes = [i32, P(i32), P(i32), i32, P(i32)]
            L.or_energy_terms.restype = i64
            L.or_energy_terms.argtypes = [i32, P(i32), i32, i32, P(ct.c_uint8), P(i64), P(i64), P(i64)]
            L.or_dense_qubo.restype = None
            L.or_dense_qubo.argtypes = [i32, P(i32), i32, i32, P(i32), P(i64)]
            L.or_energy_terms_weighted.restype = i64
            L.or_energy_terms_weighted.argtypes = [i32, P(i32), i32, P(i32), P(ct.c_uint8)]
            L.or_dense_qubo_weighted.restype = None
            L.or_dense_qubo_weighted.argtypes = [i32, P(i32), i32, P(i32), P(i32), P(i64)]
            L.or_energy_dense.restype = i64
            L.or_energy_dense.argtypes = [i64, P(i32), i64, P(ct.c_uint8)]
            L.or_philox4x32_10.restype = None
            L.or_philox4x32_10.argtypes = [P(ct.c_uint32), P(ct.c_uint32), P(ct.c_uint32)]
            L.or_temperature.restype = dbl
            L.or_temperature.argtypes = [i32, dbl, dbl, i32]
            L.or_thresholds.restype = i32
            L.or_thresholds.argtypes = [dbl, P(ct.c_uint32), i32]
            L.or_anneal_structured.restype = i32
            L.or_anneal_structured.argtypes = [
                i32, P(i32), i32, i32, i32, i32, dbl, dbl, i32, i32, u64, i32, P(i32),
                P(ct.c_uint8), P(ct.c_uint8), P(i64), P(i64), P(i64), i32]
            L.or_anneal_dense.restype = i32
            L.or_anneal_dense.argtypes = [
                i64, P(i32), i64, P(ct.c_uint8), P(ct.c_uint8), i32, i32, dbl, dbl, i32, i32,
                u64, i32, P(i32), P(ct.c_uint8), P(ct.c_uint8), P(i64), P(i64), P(i64), i32]
            L.or_delta_at.restype = i64
            L.or_delta_at.argtypes = [i32, i32, P(i32), i32, i32, i64, P(i32), P(ct.c_uint8), i64]
            L.or_decode.restype = i32
            L.or_decode.argtypes = [i32, P(i32), P(ct.c_uint8), P(i32), P(i64)]
            _lib = L
    return _lib


# --------------------------------------------------------------------------- field
def cells(rows: int, cols: int, free_mask, start: int):
    """Section II: free cells in row-major order -> (cell_r, cell_c, start_cell)."""
    m = None if free_mask is None else np.ascontiguousarray(free_mask, dtype=np.uint8).reshape(-1)
    cr = np.zeros(rows * cols, np.int32)
    cc = np.zeros(rows * cols, np.int32)
    sc = np.zeros(1, np.int32)
    C = lib().or_cells(rows, cols, _p(m, ct.c_uint8), start, _p(cr, ct.c_int32), _p(cc, ct.c_int32),
                       _p(sc, ct.c_int32))
    return cr[:C].copy(), cc[:C].copy(), int(sc[0])


def round_scaled_sqrt(q: int, scale: int) -> int:
    return int(lib().or_round_scaled_sqrt(int(q), int(scale)))


def distances(cell_r, cell_c, scale: int = 100):
    cr = np.ascontiguousarray(cell_r, np.int32)
    cc = np.ascontiguousarray(cell_c, np.int32)
    C = len(cr)
    d = np.zeros((C, C), np.int32)
    lib().or_distances(C, _p(cr, ct.c_int32), _p(cc, ct.c_int32), scale, _p(d, ct.c_int32))
    return d


class Problem:
    """A field turned into the path QUBO's structured terms (Sections II, III-B)."""

    def __init__(self, rows, cols, free_mask=None, start=0, A=None, B=1, scale=100):
        self.rows, self.cols = rows, cols
        self.cell_r, self.cell_c, self.start_cell = cells(rows, cols, free_mask, start)
        if self.start_cell < 0:
            raise ValueError("start cell is not free")
        self.C = len(self.cell_r)
        self.n = self.C * self.C
        self.d = distances(self.cell_r, self.cell_c, scale)
        self.max_d = int(self.d.max()) if self.C > 0 else 0
        self.A = int(2 * self.max_d if A is None else A)
        self.B = int(B)

    def energy(self, x):
        return energy_terms(self.d, self.A, self.B, x)[0]

    def dense(self):
        return dense_qubo(self.d, self.A, self.B)

    def frozen(self):
        """Reading R5 as masks over k = t*C + i."""
        C, s = self.C, self.start_cell
        fr = np.zeros((C, C), np.uint8)
        fr[0, :] = 1
        fr[:, s] = 1
        fv = np.zeros((C, C), np.uint8)
        fv[0, s] = 1
        return fr.reshape(-1), fv.reshape(-1)


# --------------------------------------------------------------------------- energy
def energy_terms(d, A, B, x):
    """Eqs. 3-6 -> (E, H_dist, H_visit, H_time)."""
    d = np.ascontiguousarray(d, np.int32)
    C = d.shape[0]
    x = np.ascontiguousarray(x, np.uint8).reshape(-1)
    assert x.size == C * C
    hd, hv, ht = (np.zeros(1, np.int64) for _ in range(3))
    e = lib().or_energy_terms(C, _p(d, ct.c_int32), int(A), int(B), _p(x, ct.c_uint8),
                              _p(hd, ct.c_int64), _p(hv, ct.c_int64), _p(ht, ct.c_int64))
    return int(e), int(hd[0]), int(hv[0]), int(ht[0])


def dense_qubo(d, A, B):
    d = np.ascontiguousarray(d, np.int32)
    C = d.shape[0]
    n = C * C
    S = np.zeros((n, n), np.int32)
    c0 = np.zeros(1, np.int64)
    lib().or_dense_qubo(C, _p(d, ct.c_int32), int(A), int(B), _p(S, ct.c_int32), _p(c0, ct.c_int64))
    return S, int(c0[0])


def energy_terms_weighted(d, A, w, x):
    """Reading R9: Eq. 6 with leg weights w[0..C-2] on the distance term."""
    d = np.ascontiguousarray(d, np.int32)
    C = d.shape[0]
    w = np.ascontiguousarray(w, np.int32)
    assert w.size == C - 1
    x = np.ascontiguousarray(x, np.uint8).reshape(-1)
    assert x.size == C * C
    return int(lib().or_energy_terms_weighted(C, _p(d, ct.c_int32), int(A), _p(w, ct.c_int32), _p(x, ct.c_uint8)))


def dense_qubo_weighted(d, A, w):
    """Reading R9: the dense form of energy_terms_weighted -> (S, c0)."""
    d = np.ascontiguousarray(d, np.int32)
    C = d.shape[0]
    w = np.ascontiguousarray(w, np.int32)
    assert w.size == C - 1
    n = C * C
    S = np.zeros((n, n), np.int32)
    c0 = np.zeros(1, np.int64)
    lib().or_dense_qubo_weighted(C, _p(d, ct.c_int32), int(A), _p(w, ct.c_int32), _p(S, ct.c_int32),
                                 _p(c0, ct.c_int64))
    return S, int(c0[0])


def energy_dense(S, c0, x):
    S = np.ascontiguousarray(S, np.int32)
    x = np.ascontiguousarray(x, np.uint8).reshape(-1)
    return int(lib().or_energy_dense(S.shape[0], _p(S, ct.c_int32), int(c0), _p(x, ct.c_uint8)))


# --------------------------------------------------------------------------- rng / schedule
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_p(c, ct.c_uint32), _p(k, ct.c_uint32), _p(out, ct.c_uint32))
    return out


def temperature(n_sweeps, T0, T1, s):
    return float(lib().or_temperature(n_sweeps, T0, T1, s))


def thresholds(T):
    n = lib().or_thresholds(float(T), None, 0)
    out = np.zeros(n, np.uint32)
    lib().or_thresholds(float(T), _p(out, ct.c_uint32), n)
    return out


# --------------------------------------------------------------------------- anneal
class Result:
    def __init__(self, states, energies, best, accepts):
        self.states, self.energies, self.best, self.accepts = states, energies, best, accepts


def _threads(n_threads):
    return int(n_threads or os.cpu_count() or 1)


def anneal_structured(prob: Problem, replicas, n_sweeps, T0=1e3, T1=1.0, seed=1,
                      sweep_begin=0, sweep_end=None, init_states=None, n_threads=None):
    """Sequential-sweep Metropolis on the structured form.  `replicas` is a count
    (indices 0..R-1) or an explicit list of global replica indices."""
    idx = np.arange(replicas, dtype=np.int32) if np.isscalar(replicas) else np.asarray(replicas, np.int32)
    R = len(idx)
    n = prob.n
    se = n_sweeps if sweep_end is None else sweep_end
    st = np.zeros((R, n), np.uint8)
    E = np.zeros(R, np.int64)
    best = np.zeros(R, np.int64)
    acc = np.zeros(R, np.int64)
    init = None if init_states is None else np.ascontiguousarray(init_states, np.uint8).reshape(R, n)
    rc = lib().or_anneal_structured(
        prob.C, _p(np.ascontiguousarray(prob.d, np.int32), ct.c_int32), prob.A, prob.B, prob.start_cell,
        n_sweeps, float(T0), float(T1), sweep_begin, se, seed, R, _p(idx, ct.c_int32),
        _p(init, ct.c_uint8), _p(st, ct.c_uint8), _p(E, ct.c_int64), _p(best, ct.c_int64),
        _p(acc, ct.c_int64), _threads(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle anneal failed: {rc}")
    return Result(st, E, best, acc)


def anneal_dense(S, c0, replicas, n_sweeps, T0=1e3, T1=1.0, seed=1, frozen=None, frozen_val=None,
                 C=0, sweep_begin=0, sweep_end=None, init_states=None, n_threads=None):
    S = np.ascontiguousarray(S, np.int32)
    n = S.shape[0]
    idx = np.arange(replicas, dtype=np.int32) if np.isscalar(replicas) else np.asarray(replicas, np.int32)
    R = len(idx)
    se = n_sweeps if sweep_end is None else sweep_end
    st = np.zeros((R, n), np.uint8)
    E = np.zeros(R, np.int64)
    best = np.zeros(R, np.int64)
    acc = np.zeros(R, np.int64)
    fr = None if frozen is None else np.ascontiguousarray(frozen, np.uint8)
    fv = None if frozen_val is None else np.ascontiguousarray(frozen_val, np.uint8)
    init = None if init_states is None else np.ascontiguousarray(init_states, np.uint8).reshape(R, n)
    rc = lib().or_anneal_dense(
        n, _p(S, ct.c_int32), int(c0), _p(fr, ct.c_uint8), _p(fv, ct.c_uint8), int(C), n_sweeps,
        float(T0), float(T1), sweep_begin, se, seed, R, _p(idx, ct.c_int32), _p(init, ct.c_uint8),
        _p(st, ct.c_uint8), _p(E, ct.c_int64), _p(best, ct.c_int64), _p(acc, ct.c_int64),
        _threads(n_threads))
    if rc != 0:
        raise RuntimeError(f"oracle anneal failed: {rc}")
    return Result(st, E, best, acc)


def delta_path(d, A, B, x, k):
    """dE of flipping k in the structured form, from the sweep's formula."""
    d = np.ascontiguousarray(d, np.int32)
    x = np.ascontiguousarray(x, np.uint8).reshape(-1)
    return int(lib().or_delta_at(1, d.shape[0], _p(d, ct.c_int32), int(A), int(B), 0, None,
                                 _p(x, ct.c_uint8), int(k)))


def delta_dense(S, x, k):
    S = np.ascontiguousarray(S, np.int32)
    x = np.ascontiguousarray(x, np.uint8).reshape(-1)
    return int(lib().or_delta_at(0, 0, None, 0, 0, S.shape[0], _p(S, ct.c_int32),
                                 _p(x, ct.c_uint8), int(k)))


def decode(d, x):
    """Algorithm 1 last step -> (path, length) or None when infeasible."""
    d = np.ascontiguousarray(d, np.int32)
    C = d.shape[0]
    x = np.ascontiguousarray(x, np.uint8).reshape(-1)
    path = np.zeros(C, np.int32)
    L = np.zeros(1, np.int64)
    rc = lib().or_decode(C, _p(d, ct.c_int32), _p(x, ct.c_uint8), _p(path, ct.c_int32), _p(L, ct.c_int64))
    return None if rc else (path, int(L[0]))
