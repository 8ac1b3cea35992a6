"""Pins of the replica-exchange reference (oracle/pt_ref.py) -- no GPU.

* The exchange table encodes the textbook acceptance probability
  min(1, exp((1/T_m - 1/T_{m+1}) (E_a - E_b))), written here with inverse
  temperatures (not with the effective temperature the reference uses).
* Stationarity: on a 16-state path QUBO, every level of the ladder samples
  the exact Boltzmann distribution at its temperature (chi-square over many
  independent groups); a run with the trade rule reversed (planted on the
  CPU, in the reference) fails the same test, so the test sees the rule.
* Invariants of the bookkeeping: each group's owners are a permutation and
  agree with the levels; trades per pair are counted.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
from oracle import pt_ref


def test_exchange_table_is_the_acceptance_probability():
    for (T_lo, T_hi, M) in [(1.0, 1000.0, 8), (5.0, 60.0, 3), (50.0, 800.0, 4)]:
        T = pt_ref.ladder(M, T_lo, T_hi)
        assert T[0] == pytest.approx(T_lo) and T[-1] == pytest.approx(T_hi)
        for m in range(M - 1):
            tab = oracle.thresholds(pt_ref.exchange_temperature(T[m], T[m + 1]))
            dbeta = 1.0 / T[m] - 1.0 / T[m + 1]
            for X in [1, 2, 7, len(tab) // 3, len(tab) - 1]:
                p = math.exp(-dbeta * X)
                assert abs(int(tab[X]) - p * 2.0 ** 32) <= 1.0 + 1e-9 * p * 2.0 ** 32
            assert math.exp(-dbeta * len(tab)) * 2.0 ** 32 < 1.0 + 1e-6


def tiny_problem():
    # 1 x 3 strip from cell 0: (C-1)^2 = 4 free variables, 16 states
    return oracle.Problem(1, 3, None, 0)


def exact_boltzmann(P, T):
    """Probabilities of the 16 states (free variables in increasing k) at T."""
    C = P.C
    free = [k for k in range(C * C) if k // C != 0 and k % C != P.start_cell]
    E = []
    for bits in itertools.product([0, 1], repeat=len(free)):
        x = np.zeros(C * C, np.uint8)
        x[P.start_cell] = 1
        for k, b in zip(free, bits):
            x[k] = b
        E.append(P.energy(x))
    E = np.array(E, np.float64)
    w = np.exp(-(E - E.min()) / T)
    return free, w / w.sum()


def state_index(x, free):
    return int(sum(int(x[k]) << (len(free) - 1 - j) for j, k in enumerate(free)))


def chi2_per_level(out, P, G, M, T):
    free, _ = exact_boltzmann(P, 1.0)
    stats = []
    for m in range(M):
        _, p = exact_boltzmann(P, T[m])
        counts = np.zeros(len(p))
        for r in np.nonzero(out["levels"] == m)[0]:
            counts[state_index(out["states"][r], free)] += 1
        assert counts.sum() == G
        exp = p * G
        keep = exp >= 5
        chi2 = (((counts - exp) ** 2 / exp)[keep]).sum() + 0.0
        lumped = counts[~keep].sum()
        if (~keep).any():
            chi2 += (lumped - exp[~keep].sum()) ** 2 / max(exp[~keep].sum(), 1e-9)
        dof = int(keep.sum()) + (1 if (~keep).any() else 0) - 1
        stats.append((chi2, dof))
    return stats


def run_tiny():
    P = tiny_problem()
    G, M, T_lo, T_hi = 3000, 4, 60.0, 900.0
    out = pt_ref.anneal_pt(P, G, M, T_lo, T_hi, I=1, rounds=80, seed=77)
    return P, G, M, pt_ref.ladder(M, T_lo, T_hi), out


def test_levels_sample_boltzmann():
    P, G, M, T, out = run_tiny()
    for chi2, dof in chi2_per_level(out, P, G, M, T):
        # 99.9% quantile of chi-square (Wilson-Hilferty), generous for dof <= 15
        z = 3.09
        crit = dof * (1 - 2 / (9 * dof) + z * math.sqrt(2 / (9 * dof))) ** 3
        assert chi2 < crit, (chi2, dof, crit)
    assert out["swaps"].sum() > 0


def test_reversed_trade_rule_is_detected():
    """Plant the reverse rule (accept iff X >= 0 or by the table on -X) in the
    reference: the cold levels then hold the high-energy states and the
    chi-square test of the coldest level fails."""
    orig = oracle.philox4x32_10

    def flipped_anneal(prob, G, M, T_lo, T_hi, I, rounds, seed):
        R = G * M
        T = pt_ref.ladder(M, T_lo, T_hi)
        xtab = [oracle.thresholds(pt_ref.exchange_temperature(T[m], T[m + 1])) for m in range(M - 1)]
        key = np.array([seed, 0], np.uint32)
        level = [r % M for r in range(R)]
        owner = list(range(R))
        states = np.zeros((R, prob.n), np.uint8)
        E = np.zeros(R, np.int64)
        for e in range(rounds):
            for m in range(M):
                idx = np.array([r for r in range(R) if level[r] == m], np.int32)
                res = oracle.anneal_structured(prob, idx, I * rounds, T0=T[m], T1=T[m], seed=seed,
                                               sweep_begin=e * I, sweep_end=(e + 1) * I,
                                               init_states=states[idx] if e else None)
                states[idx], E[idx] = res.states, res.energies
            for g in range(G):
                for m in range(e % 2, M - 1, 2):
                    a, b = owner[g * M + m], owner[g * M + m + 1]
                    X = -(int(E[b]) - int(E[a]))  # planted mistake: sign of X reversed
                    take = X <= 0 or (X < len(xtab[m]) and int(orig([m, e, g, pt_ref.PT_TAG], key)[0]) < int(xtab[m][X]))
                    if take:
                        owner[g * M + m], owner[g * M + m + 1] = b, a
                        level[a], level[b] = m + 1, m
        return dict(states=states, levels=np.array(level))

    P = tiny_problem()
    G, M, T_lo, T_hi = 3000, 4, 60.0, 900.0
    out = flipped_anneal(P, G, M, T_lo, T_hi, 1, 80, 77)
    chi2, dof = chi2_per_level(out, P, G, M, pt_ref.ladder(M, T_lo, T_hi))[0]
    assert chi2 > 10 * dof


def test_bookkeeping_invariants():
    P = oracle.Problem(3, 3, None, 0)
    G, M = 5, 5
    out = pt_ref.anneal_pt(P, G, M, 5.0, 500.0, I=2, rounds=9, seed=3)
    lev = out["levels"]
    for g in range(G):
        assert sorted(lev[g * M:(g + 1) * M].tolist()) == list(range(M))
    assert out["swaps"].shape == (G * (M - 1),) and (out["swaps"] >= 0).all()
    # every chain's final energy is the energy of its final state
    for r in range(G * M):
        assert out["energies"][r] == P.energy(out["states"][r])
        assert out["best"][r] == oracle.E_NONE or out["best"][r] >= 800  # no path is shorter than 800
