"""Learned warm start for the annealer: data, training, seeding and the
time-to-target comparison against plain annealing.

Pipeline (all GPU work goes through the C ABI):
  1. labels   -- anneal many fields with the batched kernel; per field keep the
                 feasible final state of lowest energy; a cell's label is its
                 step in that path.
  2. training -- the per-cell MLP (qp_ws_*) with softmax cross-entropy over the
                 cell's possible steps, Adam, mini-batches of whole fields.
  3. seeding  -- features -> step logits (tcgen05 forward) -> expected step
                 per cell -> the device walk (qp_ws_walk: among the unvisited
                 cells within a slack of the nearest one, the smallest expected
                 step) -> a feasible one-hot state; a fraction of the replicas
                 start from it at a lower temperature, the rest anneal plainly
                 (fallback).
  4. judging  -- on held-out fields, against a best known path computed first
                 and independently of the arms (long plain anneals, every final
                 state repaired with 2-opt): the time (and the sweeps) until an
                 arm's best path is within 1% of it, for plain annealing, the
                 same seeding with no network (the nearest-cell walk), with an
                 untrained network and with the trained one.  Runs are split
                 into sweep segments (resumable, bit-identical to one run) so the
                 best can be read as the run proceeds.
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
                    t0_over_a=0.5, repair_passes=None, log=None):
    """-> list of (features [C,16] float32, labels [C] int32, length) for the
    fields whose anneal produced a path.  Each field is annealed with
    A = penalty(C) (None: the library default 2 max d) and T0 = t0_over_a * A
    (1e3 for the default).  The label path is the shortest feasible final
    state, or, with repair_passes set, the shortest of all final states
    repaired into paths (qp_repair_batch with that many 2-opt passes, -1 =
    until no move helps)."""
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
            if repair_passes is None:
                qpath.qp_decode_batch(h, replicas, s_, paths, lens, stream=torch.cuda.current_stream())
            else:
                qpath.qp_repair_batch(h, replicas, s_, repair_passes, paths, lens,
                                      stream=torch.cuda.current_stream())
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
# The decoder's slack.  With a slack the walk may pass over the nearest cell
# to follow the predicted order (jump an obstacle instead of stranding the
# rest of a row); on held-out 16x16 fields every slack tried (50 to 300)
# made the seeds longer, so the walk stays among the nearest cells and the
# network only breaks their ties.
WALK_SLACK = 0


def device_seed(handle, field, model=None, slack=WALK_SLACK, stream=None):
    """-> (state device uint8 [C*C], path length) of a seed decoded on the
    device: with a model, its logits -> expected steps -> the walk scored by
    them; without one, the plain nearest-cell walk (ties to the smaller id)."""
    import torch
    C = handle.info["C"]
    score = None
    if model is not None:
        X = qpath.qp_ws_features(field)
        Z = torch.empty((C, qpath.WS_STEPS), dtype=torch.float32, device="cuda")
        qpath.qp_ws_forward(model, X, Z, stream=stream)
        steps = torch.full((C,), C, dtype=torch.int32, device="cuda")
        score = qpath.qp_ws_expected_steps(Z, steps, stream=stream)
    st, _, ln = qpath.qp_ws_walk(handle, score, slack if model is not None else 0, stream=stream)
    return st, int(ln.item())


def learned_seed(model, field, handle, decode="walk", d=None):
    """-> (state uint8 [C*C], path length) of the decoded network prediction
    on the host: decode = "walk" (nearest unvisited cell, ties by the predicted
    step, qp_ws_decode_walk) or "match" (greedy max-logit matching)."""
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
            if not hasattr(init, "data_ptr"):
                init = torch.from_numpy(np.ascontiguousarray(init, np.uint8))
            self.a.copy_(init.reshape(1, n).to(self.a.device).expand(replicas, n))
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
        trace.append((t, best, max(a.done for a in arms)))
        if hit is None and best is not None and best <= target:
            hit = t
    return hit, trace[-1][1], trace


def best_known(handle, replicas=1024, n_sweeps=10000, seeds=(101,), T0=1e3, T1=1.0, repair_passes=-1,
               field=None):
    """The length the arms are judged against, fixed before any arm runs and
    independent of them: plain anneals of `replicas` chains through
    `n_sweeps` sweeps, one per seed, on the handle's QUBO and (when `field`
    is given) also at the mixing penalty (A = mixing_penalty(C), T0 = A/2,
    where the chains cross between paths more often); every final state is
    repaired into a path (2-opt until no move helps, qp_repair_batch) and the
    shortest repaired path (or best feasible energy, B = 1) is kept."""
    import torch
    runs = [(handle, T0)]
    extra = None
    if field is not None:
        extra = qpath.qp_build_qubo(field, A=mixing_penalty(handle.info["C"]))
        runs.append((extra, 0.5 * extra.info["A"]))
    best = None
    for h, t0 in runs:
        for sd in seeds:
            a = Arm(h, replicas, n_sweeps, t0, T1, sd, 0)
            a.advance(n_sweeps)
            torch.cuda.synchronize()
            for v in (a.best_length(), a.repaired_length(repair_passes)):
                if v is not None:
                    best = v if best is None else min(best, v)
    if extra is not None:
        extra.close()
    return best


ARMS = ("plain", "walk", "untrained", "learned")


def evaluate(model, fields, replicas=1024, n_sweeps=2000, seeded_fraction=0.25, T0=1e3, T1=1.0, seed_T0=None,
             segments=20, ref_sweeps=10000, ref_seeds=(101,), seed=3, penalty=None, slack=WALK_SLACK,
             untrained=None, log=None, repair_passes=None, best_known_cache=None):
    """Time (and sweeps) to within 1% of the best known path on each field, for
    four arms run on the same QUBO with the same replicas and schedule:
      plain     -- every replica anneals from zero;
      walk      -- seeded_fraction of the replicas start from the plain
                   nearest-cell walk (no network) at seed_T0 (default A/4), the
                   rest anneal plainly;
      untrained -- the same with the walk scored by an untrained network's
                   expected steps (`untrained`, default WarmStartModel(seed=1));
      learned   -- the same with the trained `model`.
    A seeded arm's clock starts before its seed is computed (features, forward,
    expected steps, walk), and the seed's own length counts as found then.  The
    best known length comes first, from best_known() (long plain anneals at
    the QUBO's penalty and at the mixing penalty, repaired), and none of the
    arms contributes to it.  With repair_passes set,
    every arm's states (and the seed) are also repaired into paths with that
    many 2-opt passes at each checkpoint, the repair on the clock.
    best_known_cache (a dict, optional) keeps each field's best known length
    across calls (keyed by the field's position and penalty)."""
    import torch
    if untrained is None:
        untrained = qpath.WarmStartModel(seed=1)
    rows = []
    s_main, s_side = torch.cuda.Stream(), torch.cuda.Stream()
    for fi, f in enumerate(fields):
        if penalty is None:
            h = qpath.qp_build_qubo(f)
            T0f = T0
        else:
            h = qpath.qp_build_qubo(f, A=penalty(int(np.asarray(f.free_mask).sum())))
            T0f = 0.5 * h.info["A"]
        info = h.info
        A = info["A"]
        sT0 = seed_T0 if seed_T0 is not None else A / 4.0
        Rs = int(round(replicas * seeded_fraction))
        # warm-up of every code path (tables, kernels, decode) before any clock starts
        Arm(h, 8, n_sweeps, T0f, T1, seed, 0).advance(1)
        Arm(h, 8, n_sweeps, sT0, T1, seed, 0).advance(1)
        device_seed(h, f, model, slack)
        torch.cuda.synchronize()
        key = (fi, penalty is None)
        if best_known_cache is not None and key in best_known_cache:
            ref = best_known_cache[key]
        else:
            ref = best_known(h, replicas, ref_sweeps, ref_seeds, T0f, T1, field=f)
            if best_known_cache is not None:
                best_known_cache[key] = ref
        target = 1.01 * ref
        row = {"field": fi, "cells": info["C"], "A": A, "T0": T0f, "seed_T0": sT0, "best_known": ref,
               "slack": slack}
        # plain arm
        plain = Arm(h, replicas, n_sweeps, T0f, T1, seed, 0, stream=s_main)
        _, pb, ptr = time_to_target(h, [plain], target, segments, repair_passes=repair_passes)
        row["plain"] = _arm_row(pb, ptr, target, None)
        for name, mdl in (("walk", None), ("untrained", untrained), ("learned", model)):
            torch.cuda.synchronize()
            t = time.perf_counter()
            state, seed_len = device_seed(h, f, mdl, slack)
            if repair_passes is not None:
                _, rep_len, _ = qpath.qp_repair_path(h, state.cpu().numpy(), repair_passes)
                seed_len = min(seed_len, rep_len)
            seeded = Arm(h, Rs, n_sweeps, sT0, T1, seed, 0, init=state, stream=s_main)
            rest = Arm(h, replicas - Rs, n_sweeps, T0f, T1, seed, Rs, stream=s_side)
            seed_time = time.perf_counter() - t
            _, b, tr = time_to_target(h, [seeded, rest], target, segments, seed_time=seed_time,
                                      repair_passes=repair_passes)
            row[name] = _arm_row(b, tr, target, (seed_time, seed_len))
        rows.append(row)
        h.close()
        if log:
            log(str(row))
    return rows


def _arm_row(final_best, trace, target, seed):
    """Time and sweeps of the first checkpoint (or the seed) within target."""
    t_hit, s_hit = None, None
    if seed is not None and seed[1] is not None and seed[1] <= target:
        t_hit, s_hit = seed[0], 0
    else:
        for tt, b, sw in trace:
            if b is not None and b <= target:
                t_hit, s_hit = tt, sw
                break
    out = {"time_to_1pct": t_hit, "sweeps_to_1pct": s_hit, "final_best": final_best,
           "final_time_s": trace[-1][0]}
    if seed is not None:
        out.update({"seed_length": seed[1], "seed_time_s": seed[0]})
    return out


def summarize(rows):
    """Per arm: fields that reached the target, mean time and sweeps to it over
    those fields, mean final gap and mean seed gap to the best known length."""
    out = {}
    for arm in ARMS:
        rs = [r[arm] for r in rows]
        hit = [x for x in rs if x["time_to_1pct"] is not None]
        gap = lambda k: [x[k] / r["best_known"] - 1.0 for x, r in zip(rs, rows) if x.get(k) is not None]
        g = gap("final_best")
        sg = gap("seed_length")
        out[arm] = {"reached": f"{len(hit)}/{len(rs)}",
                    "mean_time_s": float(np.mean([x["time_to_1pct"] for x in hit])) if hit else None,
                    "mean_sweeps": float(np.mean([x["sweeps_to_1pct"] for x in hit])) if hit else None,
                    "mean_final_gap": float(np.mean(g)) if g else None,
                    "mean_seed_gap": float(np.mean(sg)) if sg else None}
    return out


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
