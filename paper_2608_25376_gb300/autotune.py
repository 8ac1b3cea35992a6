"""Autotuner for the launch configuration of the sweeps.

Picks replicas-per-CTA for the single-field structured sweep, and
(replicas-per-CTA, CTAs, staging) for the batched persistent launch -- the
staging choice being each field's distance matrix read from L2 by every warp,
or staged in shared memory by a CTA that runs a block of that field's
replicas (QP_BATCH_D_SHARED) -- by timing each candidate on short windows of
the actual schedule (its hottest and its coldest sweeps) with CUDA events.  Results are cached in a JSON file keyed by GPU
model, kernel and field-size class (cells rounded up to a multiple of 32, plus
the replica count), so a configuration is measured once per machine.  The
choice never changes results: every configuration runs the same chains.

Cache file: $QPATH_AUTOTUNE_CACHE, else _build/autotune.json next to this file.
"""
from __future__ import annotations

import json
import math
import os
import threading

from . import qpath

_lock = threading.Lock()


def cache_path() -> str:
    return os.environ.get("QPATH_AUTOTUNE_CACHE",
                          os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json"))


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(d: dict) -> None:
    p = cache_path()
    os.makedirs(os.path.dirname(p), exist_ok=True)
    tmp = p + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, p)


def _gpu_key() -> str:
    import torch
    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return f"{p.name}/{p.multi_processor_count}sm"


def size_class(C: int) -> int:
    return int(math.ceil(C / 32.0)) * 32


def _windows(n_sweeps: int, width: int):
    w = max(1, min(width, n_sweeps // 2 if n_sweeps > 1 else 1))
    return [(0, w), (max(0, n_sweeps - w), n_sweeps)]


def _time(fn, reps: int = 2) -> float:
    import torch
    fn()  # warm
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def tune_single(h: "qpath.Handle", replicas: int, n_sweeps: int, T0: float = 1e3, T1: float = 1.0,
                candidates=(1, 2, 4, 8, 16), window: int = 40, refresh: bool = False) -> int:
    """Best replicas-per-CTA for qp_anneal_ex's structured kernel on this field size."""
    import torch
    C = h.info["C"]
    key = f"{_gpu_key()}|rows|C{size_class(C)}|R{replicas}"
    with _lock:
        cache = _load()
        if not refresh and key in cache:
            return int(cache[key]["replicas_per_cta"])
    n = h.info["n"]
    st = torch.zeros((replicas, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(replicas, dtype=torch.int64, device="cuda")
    timings = {}
    for w in candidates:
        total = 0.0
        for a, b in _windows(n_sweeps, window):
            sc = qpath.schedule(n_sweeps, T0, T1, a, b)
            total += _time(lambda: qpath.qp_anneal_ex(h, replicas, sc, 1, None, st, E, replicas_per_cta=w,
                                                      stream=torch.cuda.current_stream()))
        timings[w] = total
    best = min(timings, key=timings.get)
    with _lock:
        cache = _load()
        cache[key] = {"replicas_per_cta": best, "ms": timings}
        _store(cache)
    return best


def tune_batch(handles, replicas: int, n_sweeps: int, T0: float = 1e3, T1: float = 1.0,
               candidates_w=(2, 4, 8, 16), cta_factors=(0, 1, 2), stagings=(0, qpath.QP_BATCH_D_SHARED),
               window: int = 30, refresh: bool = False) -> tuple[int, int, int]:
    """Best (replicas_per_cta, ctas, flags) for qp_batch_create on this batch
    shape.  cta_factors: 0 = as many CTAs as fit at once, k = k CTAs per SM;
    stagings: the batch flags to try (0 = d from L2, QP_BATCH_D_SHARED = d
    staged in shared memory per CTA)."""
    import torch
    Cs = sorted(h.info["C"] for h in handles)
    key = (f"{_gpu_key()}|batch|F{len(handles)}|Cmax{size_class(Cs[-1])}|Cmed{size_class(Cs[len(Cs) // 2])}"
           f"|R{replicas}|stagings{','.join(str(x) for x in stagings)}")
    with _lock:
        cache = _load()
        if not refresh and key in cache:
            e = cache[key]
            return int(e["replicas_per_cta"]), int(e["ctas"]), int(e["flags"])
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    st = [torch.zeros((replicas, h.info["n"]), dtype=torch.uint8, device="cuda") for h in handles]
    E = [torch.zeros(replicas, dtype=torch.int64, device="cuda") for _ in handles]
    timings = {}
    for flags in stagings:
        for w in candidates_w:
            for fct in cta_factors:
                ctas = 0 if fct == 0 else fct * sms
                total = 0.0
                try:
                    for a, b in _windows(n_sweeps, window):
                        sc = qpath.schedule(n_sweeps, T0, T1, a, b)
                        bt = qpath.qp_batch_create(handles, replicas, sc, 1, st, E, replicas_per_cta=w, ctas=ctas,
                                                   flags=flags)
                        total += _time(lambda: bt.run(torch.cuda.current_stream()))
                        bt.close()
                except qpath.QpError:
                    continue
                timings[f"{w},{ctas},{flags}"] = total
    best = min(timings, key=timings.get)
    w, ctas, flags = (int(x) for x in best.split(","))
    with _lock:
        cache = _load()
        cache[key] = {"replicas_per_cta": w, "ctas": ctas, "flags": flags, "ms": timings}
        _store(cache)
    return w, ctas, flags
