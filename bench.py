#!/usr/bin/env python3
"""Throughput benchmark of the many-replica Metropolis sweep (flip attempts/s).

One step = one pass of the hot path over one batch: anneal every replica of
the workload through all its sweeps (structured kernel) and decode every final
state into a path.  The QUBO and the threshold tables are built before the
timed region (inputs resident in HBM); the end-to-end figure (`e2e`) rebuilds
the QUBO from the host field and reads every result back to pinned host memory
inside the timed region, through the same C ABI a user calls.

Workload (default, the largest single-GPU configuration): 24x24 field, 15%
obstacles dropped by a seeded Bernoulli draw (491 cells, n = 241,081
variables), int16 distances, structured terms only, int32 dE / int64
energies, 4096 replicas x 10000 sweeps, geometric T 1e3 -> 1, seed 1.
flip attempts = R * S * (C-1)^2.  The 10x10 workload (92 cells, 1024 x 5000,
structured and dense) and the others are reported as variants.

`--impl reference` times the CPU oracle (plain C, one thread per replica) on a
bounded sample of the same workload.

Multi-GPU: replicas shard with no collective on the data path (weak scaling:
every rank anneals its own replicas, streams offset by rank); the barrier
and the max-over-ranks time reduction are the only communication.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "flip attempts/s on 1 GB300; time-to-within-1%-of-best path, learned vs plain"
UNIT = "flip attempts/s"
# algorithmic integer operations per flip attempt of the structured sweep: the
# neighbour field of a one-hot state (2 adds), r' and c' (2), 2r'-1 and 2c'-1 (4),
# the A, A, B products (3), two sums (2), the sign (2), the two comparisons (2)
OPS_PER_ATTEMPT = 17
INT_LANES_PER_SM = 128
L2_FLUSH_BYTES = 512 << 20
DEFAULT_WORKLOAD = "24x24-p0.15"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-warm-start", action="store_true")
    ap.add_argument("--no-paper-protocol", action="store_true")
    ap.add_argument("--no-replica-exchange", action="store_true")
    ap.add_argument("--no-repair", action="store_true")
    ap.add_argument("--no-skip-settled", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true")
    ap.add_argument("--replicas-per-cta", type=int, default=0)
    ap.add_argument("--structured-kernel", default="rows", choices=["rows", "flat"])
    ap.add_argument("--profile-case", default=None, choices=["rows", "flat", "dense", "mlp", "batch", "repair"],
                    help="run one warm-up and one measured launch of that kernel on a sub-range of "
                         "the workload (--sweep-window, --replicas), for ncu captures")
    ap.add_argument("--sweep-window", nargs=2, type=int, default=[0, 100])
    ap.add_argument("--resume", action="store_true",
                    help="profile case: first run the chain through the sweeps before the window (one "
                         "launch), so the window starts from the chain's own state")
    ap.add_argument("--replicas", type=int, default=0)
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def kernel_source_hash():
    """Hash of the row kernel's sources; a recorded ncu figure is used only
    while it matches."""
    h = hashlib.sha256()
    for f in ["qp_sweep_rows.cu", "qp_rows.cuh", "qp_device.cuh"]:
        h.update(open(os.path.join(ROOT, "paper_2608_25376_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


PROFILE_OF = {"24x24-p0.15": "sweep_rows_24x24.md", "10x10-p0.10": "sweep_rows_10x10.md"}


def recorded_traffic(workload, kernel_tag="rows"):
    """DRAM bytes per full launch of the row kernel on `workload`, from the
    committed ncu summary, if it was taken on the current kernel source (else
    None)."""
    name = PROFILE_OF.get(workload)
    p = os.path.join(ROOT, "profiles", name) if name else None
    if not p or not os.path.exists(p):
        return None
    txt = open(p).read()
    m = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", txt)
    t = re.search(rf"{kernel_tag}_dram_bytes_per_launch_full:\s*([0-9.eE+]+)", txt)
    if not m or not t or m.group(1) != kernel_source_hash():
        return None
    return float(t.group(1))


def bytes_per_attempt(C):
    """Algorithmic bytes per flip attempt of the structured sweep (the
    bytes-per-flip model): each row t of C-1 proposals reads the distance rows
    of the hot cells of rows t-1 and t+1, 2 rows x C entries x 2 B (int16)."""
    return 2 * C * 2 / (C - 1)


def workload_config(name, f, C, n, w):
    """The `config` object of both arms' lines (identical for the same workload)."""
    return {"workload": f"{name} structured", "field": f"{f.rows}x{f.cols}", "cells": C, "variables": n,
            "replicas": w["replicas"], "sweeps": w["n_sweeps"], "schedule": "geometric 1e3->1",
            "seed": w["seed"], "attempts_per_step": w["replicas"] * w["n_sweeps"] * (C - 1) ** 2,
            "l2": "flushed between steps (512 MB write)"}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_baseline(w, P, max_seconds=20.0):
    """The oracle as it stands on this host's cores, on a bounded sample of the
    workload: about max_seconds of CPU work, one thread per replica, each
    replica through all sweeps when that fits (else a sweep prefix)."""
    import oracle
    cores = os.cpu_count() or 1
    S = w["n_sweeps"]
    probe_s = max(1, min(S, 50))
    t = time.perf_counter()
    oracle.anneal_structured(P, 1, S, seed=w["seed"], sweep_end=probe_s, n_threads=1)
    per_sweep = max((time.perf_counter() - t) / probe_s, 1e-9)
    sweeps = int(max(1, min(S, max_seconds / per_sweep)))
    if sweeps < S:
        waves = 1  # a sweep prefix already fills the budget: one replica per core
    else:
        t = time.perf_counter()  # one replica through every sweep sizes the number of waves
        oracle.anneal_structured(P, [w["replicas"] - 1], S, seed=w["seed"], n_threads=1)
        one = max(time.perf_counter() - t, 1e-9)
        waves = int(max(1, min(max(1, w["replicas"] // cores), max_seconds / one)))
    reps = cores * waves
    t = time.perf_counter()
    oracle.anneal_structured(P, reps, S, seed=w["seed"], sweep_end=sweeps, n_threads=cores)
    dt = time.perf_counter() - t
    attempts = reps * sweeps * (P.C - 1) ** 2
    return {"value": attempts / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{reps} of {w['replicas']} replicas x sweeps [0,{sweeps}) of {S}, {P.C} cells, "
                      f"one thread per replica",
            "seconds": round(dt, 2)}


def run_reference(args):
    """The oracle as it stands, on this host's cores, on the same workload and
    config as the GPU arm: each step runs `cores` replicas (one thread each)
    through a sweep prefix sized so the whole run takes a few minutes."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2608_25376_gb300 import inputs
    w = inputs.WORKLOADS[args.workload]
    f = w["field"]()
    P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start)
    cores = os.cpu_count() or 1
    S = w["n_sweeps"]
    step_s = min(10.0, max(1.0, 150.0 / max(1, args.steps)))
    t = time.perf_counter()
    oracle.anneal_structured(P, 1, S, seed=w["seed"], sweep_end=min(S, 20), n_threads=1)
    per_sweep = (time.perf_counter() - t) / min(S, 20)
    sweeps = int(max(1, min(S, step_s / max(per_sweep, 1e-9))))
    for _ in range(args.warmup):
        oracle.anneal_structured(P, cores, S, seed=w["seed"], sweep_end=min(sweeps, 5), n_threads=cores)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.anneal_structured(P, cores, S, seed=w["seed"], sweep_end=sweeps, n_threads=cores)
        times.append(time.perf_counter() - t)
    attempts = cores * sweeps * (P.C - 1) ** 2
    ms = 1e3 * statistics.mean(times)
    val = attempts / (ms / 1e3)
    sample = (f"{cores} of {w['replicas']} replicas (one thread each) x sweeps [0,{sweeps}) of {S} per step, "
              f"{P.C} cells")
    line = {"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic", "impl": "reference",
            "config": workload_config(args.workload, f, P.C, P.n, w),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def bench_batch(args, flush, stream):
    """The batched workload: 256 fields (sides 4..16, 0-20% obstacles, irregular
    boundaries, seed 2026) x 128 replicas x 2000 sweeps in one CUDA-graph launch,
    configuration from the autotuner."""
    import torch
    from paper_2608_25376_gb300 import autotune, inputs, qpath
    fields = inputs.batch(256, seed=2026)
    hs = [qpath.qp_build_qubo(f) for f in fields]
    R, S = 128, 2000
    w, ctas, bflags = autotune.tune_batch(hs, R, S)
    st = [torch.zeros((R, h.info["n"]), dtype=torch.uint8, device="cuda") for h in hs]
    E = [torch.zeros(R, dtype=torch.int64, device="cuda") for _ in hs]
    B = [torch.zeros(R, dtype=torch.int64, device="cuda") for _ in hs]
    b = qpath.qp_batch_create(hs, R, qpath.schedule(S), 1, st, E, B, replicas_per_cta=w, ctas=ctas, flags=bflags)
    attempts = sum(R * S * (h.info["C"] - 1) ** 2 for h in hs)
    with torch.cuda.stream(stream):
        b.run(stream)
        ms = []
        for k in range(2):
            flush.fill_(k)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.run(stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    m = statistics.mean(ms)
    feas = sum(int((x < qpath.E_NONE).sum().item()) for x in B)
    info = b.info
    b.close()
    Cs = [h.info["C"] for h in hs]
    return {"value": attempts / (m / 1e3), "unit": UNIT, "ms": m, "fields": len(hs), "replicas": R, "sweeps": S,
            "cells_min_median_max": [min(Cs), sorted(Cs)[len(Cs) // 2], max(Cs)], "attempts": attempts,
            "replicas_per_cta": info["replicas_per_cta"], "ctas": info["ctas"], "launch": "one CUDA graph",
            "staging": "d in shared memory per CTA" if bflags & qpath.QP_BATCH_D_SHARED else "d from L2",
            "feasible_replicas": feas}


def bench_warm_start():
    """Time to within 1% of a best known path fixed beforehand (long plain
    anneals, every final state repaired with 2-opt), on 4 held-out 16x16
    fields, 1024 replicas x 2000 sweeps per arm, 25% seeded: plain annealing,
    seeds from the nearest-cell walk alone, from the walk with an untrained
    network's tie-break, and with the trained one.  A reduced training set
    keeps the bench short: labels from 1024 seeded 8..16 fields (32 replicas x
    2000 sweeps, final states repaired), 8 epochs; the 10000-field workload is
    `python -m paper_2608_25376_gb300.warmstart`."""
    from paper_2608_25376_gb300 import inputs, qpath, warmstart
    t = time.perf_counter()
    data = warmstart.annealer_labels(inputs.fields_8_16(1024, seed=1000), replicas=32, n_sweeps=2000,
                                     repair_passes=-1)
    m = qpath.WarmStartModel(seed=1)
    losses = warmstart.train(m, data, epochs=8)
    prep = time.perf_counter() - t
    ev = inputs.fields_8_16(4, seed=999999, square=16)
    cache = {}
    out = {"metric": "seconds (and sweeps) to within 1% of the best known path; mean over the fields an arm "
                     "reached it on",
           "fields": "4 held-out 16x16 (seed 999999), A = 2 max d, 1024 replicas x 2000 sweeps per arm, 25% seeded",
           "best_known": "plain anneals (1024 replicas x 10000 sweeps) at A = 2 max d and at the mixing penalty "
                         "A = 300 + 2C, every final state repaired (2-opt); fixed before the arms run",
           "training": f"{len(data)} fields, {len(losses)} steps, loss {losses[0]:.3f} -> {losses[-1]:.3f}, "
                       f"labels+training {prep:.1f} s",
           "decoder": f"device walk, slack {warmstart.WALK_SLACK}"}
    for tag, rp in (("annealer", None), ("with_repair", -1)):
        rows = warmstart.evaluate(m, ev, replicas=1024, n_sweeps=2000, ref_sweeps=10000, repair_passes=rp,
                                  best_known_cache=cache)
        out[tag] = warmstart.summarize(rows)
    out["best_known_lengths"] = [cache[k] for k in sorted(cache)]
    return out


def bench_replica_exchange(f, flush, stream):
    """Replica exchange on the bench field: 1024 chains as 32 groups x 32
    ladder levels (T 2 -> 1000), 25 sweeps between exchange rounds, 200 rounds
    (5000 sweeps per chain, as the plain anneal).  Best path found (minimum
    best-feasible energy = length, B = 1) against the plain anneal at the same
    sweeps and at the same wall time (plain restarts with fresh seeds)."""
    import math
    import torch
    from paper_2608_25376_gb300 import qpath
    h = qpath.qp_build_qubo(f)
    n, C = h.info["n"], h.info["C"]
    G, M, I, rounds = 32, 32, 25, 200
    R = G * M
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    lv = torch.zeros(R, dtype=torch.int32, device="cuda")
    sw = torch.zeros(G * (M - 1), dtype=torch.int64, device="cuda")
    pt = qpath.pt_schedule(M, 2.0, 1000.0, I, rounds)

    def timed(fn):
        flush_l2(flush, stream, 3)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        return a.elapsed_time(b)

    qpath.qp_anneal_pt(h, G, qpath.pt_schedule(M, 2.0, 1000.0, I, 2), 1, None, st, E, B, lv, sw, stream=stream)
    pt_ms = timed(lambda: qpath.qp_anneal_pt(h, G, pt, 1, None, st, E, B, lv, sw, stream=stream))
    pt_best = int(B.min().item())
    trade = (sw.view(G, M - 1).double().mean(0) / (rounds / 2)).cpu().numpy()
    sc = qpath.schedule(I * rounds)
    plain = []
    k = 0
    spent = 0.0
    while k < 1 or spent < pt_ms:
        k += 1
        spent += timed(lambda: qpath.qp_anneal(h, R, sc, k, None, st, E, B, stream=stream))
        plain.append(int(B.min().item()))
    attempts = R * I * rounds * (C - 1) ** 2
    h.close()
    return {"config": f"{G} groups x {M} levels, T 2 -> 1000 geometric, {I} sweeps per exchange, {rounds} rounds",
            "value": attempts / (pt_ms / 1e3), "unit": UNIT, "ms": pt_ms,
            "best_length": pt_best, "plain_best_same_sweeps": plain[0],
            "plain_best_same_time": min(plain), "plain_restarts": k, "plain_ms": spent,
            "trade_rate_min_max": [float(trade.min()), float(trade.max())]}


def bench_paper_protocol():
    """The paper's evaluation protocol (Section IV-C, Table II): full M x N
    grids from a corner, the solver under a 100 ms limit.  Each grid runs the
    time-budgeted call twice (repair without and with 2-opt) after one
    untimed call that builds the schedule's tables.  The optimum is 100 (C-1):
    a serpentine exists and every step is at least one pitch."""
    from paper_2608_25376_gb300 import inputs, qpath
    rows = []
    sc = qpath.schedule(2000)
    for (M, N) in inputs.PAPER_GRIDS:
        h = qpath.qp_build_qubo(inputs.rect(M, N))
        C = M * N
        qpath.qp_anneal_timed(h, 1024, sc, 0, time_limit_ms=100.0, max_passes=0)
        row = {"grid": f"{M}x{N}", "optimum": 100 * (C - 1)}
        for tag, passes in (("annealer", 0), ("annealer+2opt", -1)):
            o = qpath.qp_anneal_timed(h, 1024, sc, 1, time_limit_ms=100.0, max_passes=passes)
            row[tag] = {"length": o["length"], "gap": o["length"] / (100 * (C - 1)) - 1.0,
                        "elapsed_ms": round(o["elapsed_ms"], 2), "rounds": o["rounds"],
                        "sweeps": o["n_sweeps"], "feasible_final_states": o["n_feasible"],
                        "status": o["status"]}
        # smallest budget in the ladder at which the repaired path is optimal
        row["ms_to_optimum_with_2opt"] = None
        for budget in (1.0, 2.0, 5.0, 10.0, 20.0, 50.0, 100.0):
            o = qpath.qp_anneal_timed(h, 1024, sc, 2, time_limit_ms=budget, max_passes=-1)
            if o["length"] == 100 * (C - 1):
                row["ms_to_optimum_with_2opt"] = {"budget_ms": budget, "elapsed_ms": round(o["elapsed_ms"], 2)}
                break
        rows.append(row)
        h.close()
    return {"protocol": "qp_anneal_timed, 100 ms limit, 1024 replicas per round, geometric 1e3->1 over "
                        "2000 sweeps, A = 2 max d, seed 1; the paper reports optimal paths in under 320 ms "
                        "on its cloud annealer (GPU model not stated)",
            "grids": rows}


def bench_repair(h, states, R, flush, stream):
    """Repair (greedy fix + 2-opt to convergence) of the step's R final states
    on the device, one warp per state; returns the timing and 8 states (host)
    for the CPU reference."""
    import torch
    from paper_2608_25376_gb300 import qpath
    C = h.info["C"]
    paths = torch.zeros((R, C), dtype=torch.int32, device="cuda")
    lens = torch.zeros(R, dtype=torch.int64, device="cuda")
    stat = torch.zeros(R, dtype=torch.int32, device="cuda")
    qpath.qp_repair_batch(h, R, states, -1, paths, lens, stat, stream=stream)
    ts = []
    for k in range(3):
        flush_l2(flush, stream, k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        qpath.qp_repair_batch(h, R, states, -1, paths, lens, stat, stream=stream)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = statistics.mean(ts)
    counts = torch.bincount(stat.long(), minlength=3).tolist()
    return ({"value": R / (ms / 1e3), "unit": "states/s", "ms": ms, "states": R, "cells": C,
             "passes": "2-opt until no move shortens the path",
             "kept_shortened_fixed": counts[:3], "mean_length": float(lens.double().mean().item()),
             "best_length": int(lens.min().item())},
            states[:8].cpu().numpy())


def cpu_other_rows(P, repair_states, with_pt):
    """The CPU references of the repair and of replica exchange, as they stand,
    on bounded samples of the 10x10 field (the variants' field)."""
    import oracle
    from oracle import pt_ref, repair_ref
    out = {}
    if repair_states is not None:
        dl = P.d.tolist()
        t0 = time.perf_counter()
        for x in repair_states:
            repair_ref.repair(x.tolist(), dl, P.C, P.start_cell, -1)
        dt = time.perf_counter() - t0
        out["repair"] = {"value": len(repair_states) / dt, "unit": "states/s", "cores": 1, "kind": "oracle",
                         "sample": f"{len(repair_states)} of the step's final states, greedy fix + 2-opt to "
                                   f"convergence, plain Python", "seconds": dt}
    if with_pt:
        G, M, I, rounds = 16, 32, 25, 10
        t0 = time.perf_counter()
        pt_ref.anneal_pt(P, G, M, 2.0, 1000.0, I, rounds, seed=1)
        dt = time.perf_counter() - t0
        out["replica_exchange"] = {"value": G * M * I * rounds * (P.C - 1) ** 2 / dt, "unit": UNIT,
                                   "cores": os.cpu_count(), "kind": "oracle",
                                   "sample": f"{G} groups x {M} levels, {rounds} rounds of {I} sweeps "
                                             f"(the variant's ladder, fewer groups and rounds)",
                                   "seconds": dt}
    return out


def flush_l2(flush, stream, k):
    """Evict L2 by a write larger than it, on `stream`, so the flush is done
    before the events recorded after it (a flush on another stream would
    overlap the timed kernel)."""
    import torch
    with torch.cuda.stream(stream):
        flush.fill_(k)


def timed_anneal(h, R, sc, seed, flush, stream, runs=2, warm=True, **kw):
    """CUDA-event times (ms, on `stream`) of `runs` calls of qp_anneal_ex after
    an optional warm-up call; L2 flushed before each."""
    import torch
    from paper_2608_25376_gb300 import qpath
    n = h.info["n"]
    st = kw.pop("states", None)
    if st is None:
        st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    acc = torch.zeros(R, dtype=torch.int64, device="cuda")
    if warm:
        qpath.qp_anneal_ex(h, R, sc, seed, None, st, E, B, accepts_out=acc, stream=stream, **kw)
    ms = []
    for k in range(runs):
        flush_l2(flush, stream, k)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        qpath.qp_anneal_ex(h, R, sc, seed, None, st, E, B, accepts_out=acc, stream=stream, **kw)
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
    return ms, st, E, B, acc


def bench_10x10(flush, stream, pk, pk_kind, skip_settled=True, repair=True):
    """The 10x10 workload (10% obstacles, 92 cells, 1024 replicas x 5000
    sweeps): the row kernel (d staged in shared memory), the dense-Q kernel
    (int16 S, 143 MB, streamed from HBM), the row kernel with settled sweeps
    skipped (same results) and the repair of the final states.  Returns the
    variant's record and 8 final states for the CPU repair reference."""
    import torch
    from paper_2608_25376_gb300 import inputs, qpath
    name = "10x10-p0.10"
    w = inputs.WORKLOADS[name]
    h = qpath.qp_build_qubo(w["field"](), flags=qpath.QP_STRUCTURED | qpath.QP_DENSE)
    n, C = h.info["n"], h.info["C"]
    R, S, seed = w["replicas"], w["n_sweeps"], w["seed"]
    sc = qpath.schedule(S)
    attempts = R * S * (C - 1) ** 2
    out = {"workload": f"{name}: {C} cells, {R} replicas x {S} sweeps", "attempts": attempts}
    ms, st, E, B, _ = timed_anneal(h, R, sc, seed, flush, stream, runs=3, kernel=qpath.QP_KERNEL_STRUCTURED)
    rows_ms = statistics.mean(ms)
    bpa = bytes_per_attempt(C)
    out["rows"] = {"value": attempts / (rows_ms / 1e3), "unit": UNIT, "kernel_ms": rows_ms,
                   "bytes_per_flip_GBps": bpa * attempts / (rows_ms / 1e3) / 1e9,
                   "traffic": recorded_traffic(name)}
    ref_E, ref_B = E.clone(), B.clone()
    dms, _, dE, dB, dacc = timed_anneal(h, R, sc, seed, flush, stream, runs=2, kernel=qpath.QP_KERNEL_DENSE)
    dm = statistics.mean(dms)
    col_bytes = float(dacc.sum().item()) * ((n + 7) // 8 * 8) * 2  # accepted flips x one int16 row of S
    out["dense"] = {"value": attempts / (dm / 1e3), "unit": UNIT, "kernel_ms": dm,
                    "column_bytes_per_launch": col_bytes, "column_GBps": col_bytes / (dm / 1e3) / 1e9,
                    "frac_of_hbm": col_bytes / (dm / 1e3) / 1e9 / pk["hbm_gbs"] if pk.get("hbm_gbs") else None,
                    "hbm_peak_GBps": pk.get("hbm_gbs"), "peak_kind": pk_kind,
                    "same_results_as_rows": bool(torch.equal(dE, ref_E) and torch.equal(dB, ref_B))}
    if skip_settled:
        sms, _, sE, sB, _ = timed_anneal(h, R, sc, seed, flush, stream, runs=3, warm=False,
                                         flags=qpath.QP_ANNEAL_SKIP_SETTLED)
        out["skip_settled"] = {"ms": statistics.mean(sms), "speedup": rows_ms / statistics.mean(sms),
                               "same_results": bool(torch.equal(sE, ref_E) and torch.equal(sB, ref_B)),
                               "note": "sweeps after a replica met no proposal with dE < len are not evaluated; "
                                       "not a headline number"}
    sample = None
    if repair:
        out["repair"], sample = bench_repair(h, st, R, flush, stream)
    h.close()
    return out, sample


def bench_4x4_dense(flush, stream):
    """The 4x4 obstacle-free grid as a dense QUBO (64 replicas x 2000 sweeps)."""
    from paper_2608_25376_gb300 import inputs, qpath
    w = inputs.WORKLOADS["4x4-dense"]
    h = qpath.qp_build_qubo(w["field"](), flags=qpath.QP_STRUCTURED | qpath.QP_DENSE)
    C = h.info["C"]
    R, S = w["replicas"], w["n_sweeps"]
    ms, _, _, B, _ = timed_anneal(h, R, qpath.schedule(S), w["seed"], flush, stream, runs=2,
                                  kernel=qpath.QP_KERNEL_DENSE)
    attempts = R * S * (C - 1) ** 2
    m = statistics.mean(ms)
    out = {"value": attempts / (m / 1e3), "unit": UNIT, "ms": m, "attempts": attempts, "kernel": "dense",
           "best_energy": int(B.min().item()), "optimum": 100 * (C - 1)}
    h.close()
    return out


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import fcntl
    from paper_2608_25376_gb300 import build as qbuild
    os.makedirs(qbuild.BUILD, exist_ok=True)
    with open(os.path.join(qbuild.BUILD, ".lock"), "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        qbuild.build()
        fcntl.flock(lk, fcntl.LOCK_UN)
    from paper_2608_25376_gb300 import inputs, qpath, shard

    w = inputs.WORKLOADS[args.workload]
    f = w["field"]()
    R, S, seed = w["replicas"], w["n_sweeps"], w["seed"]
    h = qpath.qp_build_qubo(f, flags=qpath.QP_STRUCTURED)
    info = h.info
    C, n = info["C"], info["n"]
    attempts = R * S * (C - 1) ** 2
    sc = qpath.schedule(S)
    dev = torch.device("cuda", local)
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    stream = torch.cuda.Stream(device=dev)
    states = torch.zeros((R, n), dtype=torch.uint8, device=dev)
    E = torch.zeros(R, dtype=torch.int64, device=dev)
    best = torch.zeros(R, dtype=torch.int64, device=dev)
    acc = torch.zeros(R, dtype=torch.int64, device=dev)
    paths = torch.zeros((R, C), dtype=torch.int32, device=dev)
    lens = torch.zeros(R, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    offset, _ = shard.replica_range(rank, world, R, "weak")
    rpc = args.replicas_per_cta
    skernel = qpath.QP_KERNEL_STRUCTURED if args.structured_kernel == "rows" else qpath.QP_KERNEL_STRUCTURED_FLAT

    def step():
        qpath.qp_anneal_ex(h, R, sc, seed, None, states, E, best, kernel=skernel, replicas_per_cta=rpc,
                           replica_offset=offset, accepts_out=acc, stream=stream)
        qpath.qp_decode_batch(h, R, states, paths, lens, stream=stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    torch.cuda.synchronize()

    clocks = Clocks(local)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
           torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k)  # evict L2 between timed steps (outside the events)
            ev[k][0].record(stream)
            qpath.qp_anneal_ex(h, R, sc, seed, None, states, E, best, kernel=skernel,
                               replicas_per_cta=rpc, replica_offset=offset, accepts_out=acc, stream=stream)
            ev[k][1].record(stream)
            qpath.qp_decode_batch(h, R, states, paths, lens, stream=stream)
            ev[k][2].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    anneal_ms = [a.elapsed_time(b) for a, b, _ in ev]
    ms = statistics.mean(step_ms)
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    value = world * attempts / (ms_max / 1e3)
    feasible = int((lens >= 0).sum().item())
    best_len = int(lens[lens >= 0].min().item()) if feasible else None
    best_len = shard.reduce_best(best_len if best_len is not None else np.iinfo(np.int64).max)
    best_len = None if best_len == np.iinfo(np.int64).max else best_len

    pk, pk_kind = peaks()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    ann_ms = statistics.mean(anneal_ms)
    # the bytes-per-flip roofline: algorithmic bytes per launch / kernel time
    # against the measured HBM copy rate
    bpa = bytes_per_attempt(C)
    achieved_gbs = bpa * attempts / (ann_ms / 1e3) / 1e9
    # the integer-issue view beside it
    peak_tops = sms * INT_LANES_PER_SM * sm_mhz * 1e6 / 1e12
    achieved_tops = OPS_PER_ATTEMPT * attempts / (ann_ms / 1e3) / 1e12
    d_i16 = info["max_d"] <= 32767
    Cp = (C + 7) // 8 * 8
    d_where = "shared memory" if C * Cp * 4 <= 160 * 1024 else "L2 (global memory)"
    roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                "frac": achieved_gbs / pk["hbm_gbs"] if pk.get("hbm_gbs") else None,
                "traffic": recorded_traffic(args.workload),
                "kernel": ("k_sweep_structured" if args.structured_kernel != "rows"
                           else ("k_sweep_rows_g" if 256 < C <= 512 else "k_sweep_rows")),
                "kernel_ms": ann_ms, "bytes_per_attempt": bpa,
                "algorithmic_bytes_per_launch": bpa * attempts,
                "note": (f"bytes-per-flip model: 2 distance rows x {C} int16 entries per row of {C - 1} "
                         f"proposals ({bpa:.3f} B per attempt); peak = {pk_kind} HBM copy rate; the d rows "
                         f"come from {d_where}, so DRAM moves only the tables and the states ('traffic')"),
                "alu_view": {"achieved": achieved_tops, "peak": peak_tops, "unit": "Tops/s",
                             "frac": achieved_tops / peak_tops,
                             "note": f"{OPS_PER_ATTEMPT} algorithmic int ops per attempt; peak = {sms} SMs x "
                                     f"{INT_LANES_PER_SM} lanes x {sm_mhz:.0f} MHz ({pk_kind} clock)"}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": workload_config(args.workload, f, C, n, w),
            "execution": {"parallelism": f"replicas x {world} GPU(s), no collective on the data path",
                          "sms": sms, "distances": "int16" if d_i16 else "int32"},
            "roofline": roofline,
            "gpu_launches": 2 * args.steps,
            "clocks": clk,
            "result": {"feasible_replicas": feasible, "best_length": best_len,
                       "accepts_per_attempt": float(acc.sum().item()) / attempts}}

    repair_sample = None
    if not args.no_dense and rank == 0:
        line.setdefault("variants", {})["10x10-p0.10"], repair_sample = bench_10x10(
            flush, stream, pk, pk_kind, skip_settled=not args.no_skip_settled, repair=not args.no_repair)

    if not args.no_batch and rank == 0:
        line.setdefault("variants", {})["batched"] = bench_batch(args, flush, stream)

    if not args.no_other_configs and rank == 0:
        line.setdefault("variants", {})["4x4-dense"] = bench_4x4_dense(flush, stream)

    if not args.no_replica_exchange and rank == 0:
        line.setdefault("variants", {})["replica_exchange"] = bench_replica_exchange(
            inputs.WORKLOADS["10x10-p0.10"]["field"](), flush, stream)

    if not args.no_warm_start and rank == 0:
        line["warm_start"] = bench_warm_start()

    if not args.no_paper_protocol and rank == 0:
        line["paper_protocol"] = bench_paper_protocol()

    if not args.no_e2e:
        pin_states = torch.empty((R, n), dtype=torch.uint8, pin_memory=True)
        pin_E = torch.empty(R, dtype=torch.int64, pin_memory=True)
        pin_best = torch.empty(R, dtype=torch.int64, pin_memory=True)
        pin_paths = torch.empty((R, C), dtype=torch.int32, pin_memory=True)
        pin_lens = torch.empty(R, dtype=torch.int64, pin_memory=True)
        mask = np.ascontiguousarray(f.free_mask, np.uint8)
        e_times = []
        n_e2e = max(1, min(args.steps, 2))
        for k in range(n_e2e):
            flush.fill_(k)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fld = inputs.Field(f.rows, f.cols, mask, f.start)
            h2 = qpath.qp_build_qubo(fld, flags=qpath.QP_STRUCTURED)
            qpath.qp_anneal_ex(h2, R, sc, seed, None, pin_states, pin_E, pin_best, replica_offset=offset,
                               stream=stream)
            qpath.qp_decode_batch(h2, R, pin_states, pin_paths, pin_lens, stream=stream)
            torch.cuda.synchronize()
            e_times.append(time.perf_counter() - t0)
            h2.close()
        d_bytes = C * Cp * (2 if d_i16 else 4)
        h2d = mask.nbytes + d_bytes + R * n  # field, d, the host states staged again for the decode
        d2h = R * n + 16 * R + R * C * 4 + 8 * R  # states, energies + best, paths, lengths
        em = statistics.mean(e_times)
        line["e2e"] = {"value": world * attempts / em, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": em * 1e3, "steps": n_e2e,
                       "api": "qp_build_qubo + qp_anneal_ex + qp_decode_batch on pinned host buffers"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start)
        line["cpu_baseline"] = cpu_baseline(w, P)
        f10 = inputs.WORKLOADS["10x10-p0.10"]["field"]()
        P10 = oracle.Problem(f10.rows, f10.cols, f10.free_mask, f10.start)
        line["cpu_baseline"]["other_rows"] = cpu_other_rows(P10, repair_sample, not args.no_replica_exchange)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def run_profile_case(args):
    """One warm-up and one measured launch, nothing else on the GPU."""
    import torch
    from paper_2608_25376_gb300 import build as qbuild
    qbuild.build()
    from paper_2608_25376_gb300 import inputs, qpath
    if args.profile_case == "batch":
        # the batched workload's graph (256 fields x 128 replicas; the
        # configuration the autotuner picks for it: d staged in shared memory,
        # 8 replicas per CTA on 304 CTAs) over the sweep window, replayed twice
        fields = inputs.batch(256, seed=2026)
        hs = [qpath.qp_build_qubo(f) for f in fields]
        R = 128
        a, b = args.sweep_window
        sc = qpath.schedule(2000, sweep_begin=a, sweep_end=b)
        st = [torch.zeros((R, h.info["n"]), dtype=torch.uint8, device="cuda") for h in hs]
        E = [torch.zeros(R, dtype=torch.int64, device="cuda") for _ in hs]
        B = [torch.zeros(R, dtype=torch.int64, device="cuda") for _ in hs]
        bt = qpath.qp_batch_create(hs, R, sc, 1, st, E, B, replicas_per_cta=8, ctas=304,
                                   flags=qpath.QP_BATCH_D_SHARED)
        times = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bt.run(torch.cuda.current_stream())
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        attempts = sum(R * (b - a) * (h.info["C"] - 1) ** 2 for h in hs)
        print(json.dumps({"profile_case": "batch", "fields": len(hs), "replicas": R, "sweeps": [a, b], "ms": times,
                          "attempts": attempts}))
        bt.close()
        return 0
    if args.profile_case == "repair":
        # the bench step's final states (1024 replicas of the 10x10 field after
        # 5000 sweeps), then one warm-up and one measured repair of all of them
        # (greedy fix + 2-opt to convergence)
        w = inputs.WORKLOADS[args.workload]
        h = qpath.qp_build_qubo(w["field"]())
        n, C, R = h.info["n"], h.info["C"], w["replicas"]
        st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
        E = torch.zeros(R, dtype=torch.int64, device="cuda")
        qpath.qp_anneal(h, R, qpath.schedule(w["n_sweeps"]), w["seed"], None, st, E,
                        stream=torch.cuda.current_stream())
        paths = torch.zeros((R, C), dtype=torch.int32, device="cuda")
        lens = torch.zeros(R, dtype=torch.int64, device="cuda")
        times = []
        for _ in range(2):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            qpath.qp_repair_batch(h, R, st, -1, paths, lens, stream=torch.cuda.current_stream())
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        print(json.dumps({"profile_case": "repair", "workload": args.workload, "states": R, "cells": C,
                          "ms": times, "mean_length": float(lens.double().mean().item())}))
        return 0
    if args.profile_case == "mlp":
        # one warm-up and one measured training step of the warm-start MLP on
        # 16384 cells (64 fields of 256): 11 tensor-core GEMM launches a step
        import numpy as np
        M = 16384
        rng = np.random.default_rng(0)
        X = rng.random((M, qpath.WS_FEATURES), dtype=np.float32)
        Y = rng.integers(0, qpath.WS_STEPS, M).astype(np.int32)
        T = np.full(M, qpath.WS_STEPS, np.int32)
        m = qpath.WarmStartModel(seed=1)
        times = []
        for _ in range(2):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            loss = qpath.qp_ws_train_step(m, X, Y, T, 1e-3)
            torch.cuda.synchronize()
            times.append((time.perf_counter() - t0) * 1e3)
        # forward only, fused (one launch) and layered (four GEMM launches):
        # host time of the call, logits written to device memory
        Z = torch.empty((M, qpath.WS_STEPS), dtype=torch.float32, device="cuda")
        fwd = {}
        for name, mode in (("fused", qpath.QP_WS_FORWARD_FUSED), ("layered", qpath.QP_WS_FORWARD_LAYERED)):
            qpath.qp_ws_set_forward_mode(m, mode)
            ts = []
            for _ in range(4):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                qpath.qp_ws_forward(m, X, Z)
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - t0) * 1e3)
            fwd[name] = ts
        qpath.qp_ws_set_forward_mode(m, qpath.QP_WS_FORWARD_FUSED)
        print(json.dumps({"profile_case": "mlp", "cells": M, "ms": times, "loss": loss,
                          "forward_ms": fwd, "flops_per_layer_fwd": 2 * M * 256 * 256}))
        return 0
    w = inputs.WORKLOADS[args.workload]
    f = w["field"]()
    kernel = {"rows": qpath.QP_KERNEL_STRUCTURED, "flat": qpath.QP_KERNEL_STRUCTURED_FLAT,
              "dense": qpath.QP_KERNEL_DENSE}[args.profile_case]
    flags = qpath.QP_STRUCTURED | (qpath.QP_DENSE if args.profile_case == "dense" else 0)
    h = qpath.qp_build_qubo(f, flags=flags)
    n = h.info["n"]
    R = args.replicas or w["replicas"]
    a, b = args.sweep_window
    sc = qpath.schedule(w["n_sweeps"], sweep_begin=a, sweep_end=b)
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    best = torch.zeros(R, dtype=torch.int64, device="cuda")
    init = None
    if args.resume and a > 0:
        init = torch.zeros_like(st)
        qpath.qp_anneal_ex(h, R, qpath.schedule(w["n_sweeps"], sweep_end=a), w["seed"], None, init, E, best,
                           kernel=kernel, replicas_per_cta=args.replicas_per_cta, stream=torch.cuda.current_stream())
    times = []
    for _ in range(2):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        qpath.qp_anneal_ex(h, R, sc, w["seed"], init, st, E, best, kernel=kernel,
                           replicas_per_cta=args.replicas_per_cta, stream=torch.cuda.current_stream())
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    C = h.info["C"]
    print(json.dumps({"profile_case": args.profile_case, "workload": args.workload, "replicas": R,
                      "sweeps": [a, b], "ms": times, "attempts": R * (b - a) * (C - 1) ** 2}))
    return 0


def main():
    args = parse()
    if args.profile_case:
        return run_profile_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
