"""CPU reference of replica exchange (parallel tempering) -- TEST
INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module.  The paper runs many chains of its sampler in
parallel (Sections III-C, IV-A) without saying how they interact; this is
the textbook replica-exchange scheme the library offers on top of them:

* G groups of M chains; chain r = g*M + m starts at ladder level m, with
  T_m = the geometric schedule's temperature of "sweep" m of M between T_lo
  and T_hi (m = 0 coldest).
* Round e: every chain runs the sweeps [e*I, (e+1)*I) of the oracle's
  sequential Metropolis sweep at the constant temperature of its level (the
  sweep index still numbers the random draws), then the level pairs
  (m, m+1) for m = e mod 2, m+2, ... of every group try to trade.  With a
  the chain at m, b the chain at m+1 and X = E_b - E_a, the trade happens
  iff X <= 0 or (X < len and u < thr[X]), thr = the Metropolis threshold
  table at T_m T_{m+1} / (T_{m+1} - T_m), so its probability is
  min(1, exp((1/T_m - 1/T_{m+1}) (E_a - E_b))); u is word 0 of
  Philox4x32-10 at counter (m, e, g, 0x50545843) under the run's key.

The sweeps at a fixed temperature are the oracle's own anneal with T0 = T1
= T_m over the round's sweep window (T0 (T1/T0)^x is T0 exactly when
T1 = T0).  The exchange step is plain Python below.
"""
from __future__ import annotations

import numpy as np

import oracle

PT_TAG = 0x50545843


def ladder(M, T_lo, T_hi):
    return [oracle.temperature(M, T_lo, T_hi, m) for m in range(M)]


def exchange_temperature(Tm, Tn):
    return Tm * Tn / (Tn - Tm)


def anneal_pt(prob, G, M, T_lo, T_hi, I, rounds, seed, init_states=None):
    """-> dict(states, energies, best, levels, swaps) by chain, as the library
    returns them."""
    R = G * M
    n = prob.n
    T = ladder(M, T_lo, T_hi)
    xtab = [oracle.thresholds(exchange_temperature(T[m], T[m + 1])) for m in range(M - 1)]
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)
    level = [r % M for r in range(R)]
    owner = list(range(R))  # owner[g*M + m] = chain at level m of group g
    states = np.zeros((R, n), np.uint8) if init_states is None else np.array(init_states, np.uint8).reshape(R, n)
    energies = np.zeros(R, np.int64)
    best = np.full(R, oracle.E_NONE, np.int64)
    swaps = np.zeros((G, M - 1), np.int64)
    total = I * rounds
    for e in range(rounds):
        # sweeps of this round: chains grouped by their level's temperature
        for m in range(M):
            idx = np.array([r for r in range(R) if level[r] == m], np.int32)
            if len(idx) == 0:
                continue
            init = states[idx] if (e > 0 or init_states is not None) else None
            res = oracle.anneal_structured(prob, idx, total, T0=T[m], T1=T[m], seed=seed,
                                           sweep_begin=e * I, sweep_end=(e + 1) * I, init_states=init)
            states[idx] = res.states
            energies[idx] = res.energies
            best[idx] = np.minimum(best[idx], res.best)
        # exchanges
        for g in range(G):
            for m in range(e % 2, M - 1, 2):
                a, b = owner[g * M + m], owner[g * M + m + 1]
                X = int(energies[b]) - int(energies[a])
                take = X <= 0
                if not take and X < len(xtab[m]):
                    u = oracle.philox4x32_10([m, e, g, PT_TAG], key)[0]
                    take = int(u) < int(xtab[m][X])
                if take:
                    owner[g * M + m], owner[g * M + m + 1] = b, a
                    level[a], level[b] = m + 1, m
                    swaps[g, m] += 1
    return dict(states=states, energies=energies, best=best, levels=np.array(level, np.int32),
                swaps=swaps.reshape(-1))
