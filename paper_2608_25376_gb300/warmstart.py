"""Learned warm start for the annealer: data, training, seeding and the
time-to-target comparison against plain annealing.

Pipeline (all GPU work goes through the C ABI):
  1. labels   -- anneal many fields with the batched kernel; per field keep the
                 feasible final state of lowest energy; a cell's label is its
                 step in that path.
  2. training -- the per-cell MLP (qp_ws_*) with softmax cross-entropy over the
                 cell's possible steps, Adam, mini-batches of whole fields.
  3. seeding  -- features -> step logits (tcgen05 forward) -> greedy decode ->
                 a feasible one-hot state; a fraction of the replicas start from
                 it at a lower temperature, the rest anneal plainly (fallback).
  4. judging  -- time until the best feasible path found is within 1% of the
                 best known path, learned arm vs plain arm, on held-out fields;
                 runs are split into sweep segments (resumable, bit-identical to
                 one run) so the best can be read as the run proceeds.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs, qpath


def start_cell(field) -> int:
    m = np.asarray(field.free_mask, np.uint8).reshape(-1)
    return int(m[:field.start].sum())


def mixing_penalty(C: int) -> int:
    """A penalty weight near the smallest one at which most replicas still end
    feasible (about 300 + 2C at scale 100, measured on 57- to 240-cell fields):
    the chain then crosses between paths far more often than at A = 2 max d
    and finds paths 2x shorter.  Used to produce training labels."""
    return 300 + 2 * int(C)


# ----------------------------------------------------------------------------- 1. labels
def annealer_labels(fields, replicas=32, n_sweeps=2000, seed=11, chunk=256, penalty=mixing_penalty,
                    t0_over_a=0.5, log=None):
    """-> list of (features [C,16] float32, labels [C] int32, length) for the
    fields whose anneal produced a feasible final state.  Each field is
    annealed with A = penalty(C) (None: the library default 2 max d) and
    T0 = t0_over_a * A (1e3 for the default)."""
    import torch
    out = []
    for c0 in range(0, len(fields), chunk):
        part = fields[c0:c0 + chunk]
        if penalty is None:
            hs = [qpath.qp_build_qubo(f) for f in part]
            sc = qpath.schedule(n_sweeps)
        else:
            Cs = [int(np.asarray(f.free_mask).sum()) for f in part]
            hs = [qpath.qp_build_qubo(f, A=penalty(c)) for f, c in zip(part, Cs)]
            # one schedule per chunk: T0 from the chunk's median penalty
            sc = qpath.schedule(n_sweeps, t0_over_a * float(np.median([penalty(c) for c in Cs])), 1.0)
        st = [torch.zeros((replicas, h.info["n"]), dtype=torch.uint8, device="cuda") for h in hs]
        E = [torch.zeros(replicas, dtype=torch.int64, device="cuda") for _ in hs]
        qpath.qp_anneal_batch(hs, replicas, sc, seed + c0, st, E, None, stream=torch.cuda.current_stream())
        for f, h, s_, e_ in zip(part, hs, st, E):
            C = h.info["C"]
            paths = torch.zeros((replicas, C), dtype=torch.int32, device="cuda")
            lens = torch.zeros(replicas, dtype=torch.int64, device="cuda")
            qpath.qp_decode_batch(h, replicas, s_, paths, lens, stream=torch.cuda.current_stream())
            lens = lens.cpu().numpy()
            ok = np.flatnonzero(lens >= 0)
            if ok.size == 0:
                continue
            r = ok[np.argmin(lens[ok])]
            path = paths[r].cpu().numpy()
            lab = np.empty(C, np.int32)
            lab[path] = np.arange(C, dtype=np.int32)
            out.append((qpath.qp_ws_features(f), lab, int(lens[r])))
        if log:
            log(f"labels: {min(c0 + chunk, len(fields))}/{len(fields)} fields, kept {len(out)}")
    return out


# ----------------------------------------------------------------------------- 2. training
def train(model, data, epochs=4, fields_per_step=64, lr=1e-3, seed=0, log=None):
    """Adam with a cosine learning-rate decay; returns the loss of every step."""
    rng = np.random.default_rng(seed)
    n = len(data)
    steps_total = epochs * ((n + fields_per_step - 1) // fields_per_step)
    losses, k = [], 0
    for ep in range(epochs):
        order = rng.permutation(n)
        for b0 in range(0, n, fields_per_step):
            idx = order[b0:b0 + fields_per_step]
            X = np.concatenate([data[i][0] for i in idx])
            Y = np.concatenate([data[i][1] for i in idx])
            T = np.concatenate([np.full(len(data[i][1]), len(data[i][1]), np.int32) for i in idx])
            lr_k = lr * 0.5 * (1.0 + np.cos(np.pi * k / max(1, steps_total)))
            losses.append(qpath.qp_ws_train_step(model, X, Y, T, float(max(lr_k, lr * 0.02))))
            k += 1
        if log:
            log(f"epoch {ep}: loss {np.mean(losses[-max(1, n // fields_per_step):]):.4f}")
    return losses


# ----------------------------------------------------------------------------- 3. seeding
def learned_seed(model, field, handle, decode="walk", d=None):
    """-> (state uint8 [C*C], path length) of the decoded network prediction.
    decode = "walk": nearest unvisited cell, ties by the predicted step;
    "match": greedy max-logit matching of cells to steps."""
    if decode == "walk":
        d = qpath.qp_export_dist(handle) if d is None else d
        state, _ = qpath.qp_ws_infer(model, field, d)
    else:
        state, _ = qpath.qp_ws_infer(model, field, None)
    dec = qpath.qp_decode_path(handle, state)
    return state, dec[1]


# ----------------------------------------------------------------------------- 4. judging
class Arm:
    """A group of replicas annealed in sweep segments (resume = one run)."""

    def __init__(self, handle, replicas, n_sweeps, T0, T1, seed, offset, init=None, stream=None):
        import torch
        self.h, self.R, self.S = handle, replicas, n_sweeps
        self.T0, self.T1, self.seed, self.offset = T0, T1, seed, offset
        n = handle.info["n"]
        self.stream = stream
        self.a = torch.zeros((replicas, n), dtype=torch.uint8, device="cuda")
        self.b = torch.zeros_like(self.a)
        if init is not None:
            self.a.copy_(torch.from_numpy(np.broadcast_to(init, (replicas, n)).copy()))
            self.has_init = True
        else:
            self.has_init = False
        self.E = torch.zeros(replicas, dtype=torch.int64, device="cuda")
        self.best = torch.full((replicas,), qpath.E_NONE, dtype=torch.int64, device="cuda")
        self.seg_best = torch.zeros_like(self.best)
        self.done = 0

    def advance(self, sweeps):
        import torch
        a, b = self.done, min(self.S, self.done + sweeps)
        if a >= b:
            return
        sc = qpath.schedule(self.S, self.T0, self.T1, a, b)
        init = self.a if (self.has_init or a > 0) else None
        qpath.qp_anneal_ex(self.h, self.R, sc, self.seed, init, self.b, self.E, self.seg_best,
                           replica_offset=self.offset, stream=self.stream)
        with torch.cuda.stream(self.stream):
            torch.minimum(self.best, self.seg_best, out=self.best)
        self.a, self.b = self.b, self.a
        self.done = b

    def best_length(self, B=1):
        v = int(self.best.min().item())
        return None if v == qpath.E_NONE else v // B

    def repaired_length(self, passes=-1):
        """Shortest path over the replicas' current states after the repair
        (greedy fix + 2-opt, qp_repair_batch), kept as a running minimum."""
        import torch
        C = self.h.info["C"]
        paths = torch.empty((self.R, C), dtype=torch.int32, device="cuda")
        lens = torch.empty(self.R, dtype=torch.int64, device="cuda")
        qpath.qp_repair_batch(self.h, self.R, self.a, passes, paths, lens, stream=self.stream)
        if self.stream is not None:
            self.stream.synchronize()
        v = int(lens.min().item())
        self.best_rep = min(getattr(self, "best_rep", v), v)
        return self.best_rep


def time_to_target(handle, arms, target, segments, seed_time=0.0, repair_passes=None):
    """Advance every arm segment by segment (arms run concurrently, one stream
    each); -> (seconds until the best length <= target or None, final best,
    trace [(seconds, best)]).  With repair_passes set, an arm's best also
    counts its current states repaired into paths (the repair is on the
    clock)."""
    import torch
    t0 = time.perf_counter() - seed_time
    trace, hit = [], None
    total = max(a.S for a in arms)
    per = max(1, total // segments)

    def arm_best(a):
        b = a.best_length()
        if repair_passes is None:
            return b
        r = a.repaired_length(repair_passes)
        return r if b is None else min(b, r)

    while any(a.done < a.S for a in arms):
        for a in arms:
            a.advance(per)
        torch.cuda.synchronize()
        bests = [arm_best(a) for a in arms]
        best = min([b for b in bests if b is not None], default=None)
        t = time.perf_counter() - t0
        trace.append((t, best))
        if hit is None and best is not None and best <= target:
            hit = t
    return hit, trace[-1][1], trace


def evaluate(model, fields, replicas=1024, n_sweeps=2000, seeded_fraction=0.25, T0=1e3, T1=1.0,
             seed_T0=None, segments=20, ref_sweeps=10000, seed=3, penalty=None, decode="walk", log=None,
             repair_passes=None):
    """Time-to-within-1% on each field, learned arm vs plain arm.

    best known = min over: a long plain reference run (ref_sweeps), the plain
    arm, the learned arm (its seed included).  Learned arm: seeded_fraction of
    the replicas start from the decoded prediction at seed_T0 (default A/4),
    the rest anneal plainly; its clock includes features, forward and decode.
    With repair_passes set, every arm (the reference run and the seed too) is
    also judged by its states repaired into paths with that many 2-opt passes
    (qp_repair_batch; -1 = until no move helps), the repair on the clock."""
    import torch
    rows = []
    s_main, s_side = torch.cuda.Stream(), torch.cuda.Stream()
    for fi, f in enumerate(fields):
        if penalty is None:
            h = qpath.qp_build_qubo(f)
        else:
            h = qpath.qp_build_qubo(f, A=penalty(int(np.asarray(f.free_mask).sum())))
            T0 = 0.5 * h.info["A"]
        info = h.info
        A = info["A"]
        sT0 = seed_T0 if seed_T0 is not None else A / 4.0
        Rs = int(round(replicas * seeded_fraction))
        # warm-up of both code paths (tables, kernels) before any clock starts
        Arm(h, 8, n_sweeps, T0, T1, seed, 0).advance(1)
        Arm(h, 8, n_sweeps, sT0, T1, seed, 0).advance(1)
        torch.cuda.synchronize()
        # the long plain reference
        ref = Arm(h, replicas, ref_sweeps, T0, T1, seed + 7, 0, stream=s_main)
        while ref.done < ref.S:
            ref.advance(ref.S)
        torch.cuda.synchronize()
        ref_best = ref.best_length()
        if repair_passes is not None:
            r = ref.repaired_length(repair_passes)
            ref_best = r if ref_best is None else min(ref_best, r)
        # plain arm (record the trace; the target is fixed afterwards)
        plain = Arm(h, replicas, n_sweeps, T0, T1, seed, 0, stream=s_main)
        _, plain_best, plain_trace = time_to_target(h, [plain], -1, segments, repair_passes=repair_passes)
        # learned arm
        torch.cuda.synchronize()
        t = time.perf_counter()
        state, seed_len = learned_seed(model, f, h, decode=decode)
        if repair_passes is not None:
            _, rep_len, _ = qpath.qp_repair_path(h, state, repair_passes)
            seed_len = min(seed_len, rep_len)
        seeded = Arm(h, Rs, n_sweeps, sT0, T1, seed, 0, init=state, stream=s_main)
        rest = Arm(h, replicas - Rs, n_sweeps, T0, T1, seed, Rs, stream=s_side)
        seed_time = time.perf_counter() - t
        _, learned_best, learned_trace = time_to_target(h, [seeded, rest], -1, segments, seed_time=seed_time,
                                                        repair_passes=repair_passes)
        candidates = [x for x in (ref_best, plain_best, learned_best, seed_len) if x is not None]
        best_known = min(candidates)
        target = 1.01 * best_known

        def first_hit(trace, start=None):
            pts = ([(start[0], start[1])] if start else []) + list(trace)
            for tt, b in pts:
                if b is not None and b <= target:
                    return tt
            return None
        row = {"field": fi, "cells": info["C"], "A": A, "T0": T0, "seed_T0": sT0, "best_known": best_known,
               "ref_best": ref_best,
               "plain_best": plain_best, "learned_best": learned_best, "seed_length": seed_len,
               "seed_time_s": seed_time,
               "plain_time_to_1pct": first_hit(plain_trace),
               "learned_time_to_1pct": first_hit(learned_trace, (seed_time, seed_len)),
               "plain_final_time_s": plain_trace[-1][0], "learned_final_time_s": learned_trace[-1][0]}
        rows.append(row)
        if log:
            log(str(row))
    return rows


def summarize(rows):
    """Mean times over fields where the arm reached the target, and counts."""
    def stat(key):
        v = [r[key] for r in rows if r[key] is not None]
        return {"reached": len(v), "of": len(rows), "mean_s": float(np.mean(v)) if v else None}
    gap = lambda k: float(np.mean([(r[k] / r["best_known"] - 1.0) for r in rows if r[k] is not None]))
    return {"learned": stat("learned_time_to_1pct"), "plain": stat("plain_time_to_1pct"),
            "mean_gap_plain_final": gap("plain_best"), "mean_gap_learned_final": gap("learned_best"),
            "mean_gap_seed": gap("seed_length")}


def run(n_train=10000, label_replicas=64, label_sweeps=4000, epochs=8, n_eval=8, eval_side=16,
        replicas=1024, n_sweeps=2000, ref_sweeps=10000, log=print):
    """The full workload: labels from n_train seeded 8x8..16x16 fields, training,
    evaluation on n_eval held-out eval_side x eval_side fields (disjoint seeds),
    under the default penalty and under the mixing penalty."""
    t = time.perf_counter()
    fields = inputs.fields_8_16(n_train, seed=1000)
    data = annealer_labels(fields, replicas=label_replicas, n_sweeps=label_sweeps)
    t_labels = time.perf_counter() - t
    m = qpath.WarmStartModel(seed=1)
    t = time.perf_counter()
    losses = train(m, data, epochs=epochs)
    t_train = time.perf_counter() - t
    ev = inputs.fields_8_16(n_eval, seed=999999, square=eval_side)
    m0 = qpath.WarmStartModel(seed=1)
    ablation = []
    for f in ev:
        h = qpath.qp_build_qubo(f)
        ablation.append({k: learned_seed(mm, f, h, decode=dc)[1] for k, (mm, dc) in
                         {"untrained_match": (m0, "match"), "trained_match": (m, "match"),
                          "untrained_walk": (m0, "walk"), "trained_walk": (m, "walk")}.items()})
    out = {"train_fields": len(data), "label_len_per_step": float(np.mean([d[2] / (len(d[1]) - 1) for d in data])),
           "labels_s": t_labels, "train_s": t_train, "train_steps": len(losses),
           "loss_first": losses[0], "loss_last": losses[-1], "seed_ablation": ablation}
    for name, pen in (("default_A", None), ("mixing_A", mixing_penalty)):
        rows = evaluate(m, ev, replicas=replicas, n_sweeps=n_sweeps, ref_sweeps=ref_sweeps, penalty=pen)
        out[name] = {"rows": rows, "summary": summarize(rows)}
        if log:
            log(f"{name}: {summarize(rows)}")
    return out


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser(description="learned warm start: train and judge time-to-1% vs plain")
    ap.add_argument("--train-fields", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--eval-fields", type=int, default=8)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    from . import build
    build.build()
    res = run(n_train=a.train_fields, epochs=a.epochs, n_eval=a.eval_fields)
    js = json.dumps(res, indent=1, default=float)
    if a.out:
        with open(a.out, "w") as f:
            f.write(js)
    print(js)
