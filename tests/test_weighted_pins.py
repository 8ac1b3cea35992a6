"""Pins of the oracle's extended objective (reading R9 of oracle/qp_oracle.c:
the distance term of Eq. 3 with one integer weight per leg, the form Section V's
battery and pesticide objectives take here), against the unweighted forms, a
hand-worked line, brute force over every state of a small field, and brute
force over every path."""
import itertools

import numpy as np
import pytest

from paper_2608_25376_gb300 import inputs


def _d(orc, rows, cols, mask=None, scale=100):
    f = inputs.Field(rows, cols, np.ones(rows * cols, np.uint8) if mask is None else np.asarray(mask, np.uint8), 0)
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    return P.d, P.start_cell


def _state(path, C):
    x = np.zeros((C, C), np.uint8)
    for t, i in enumerate(path):
        x[t, i] = 1
    return x


def test_equal_weights_are_the_unweighted_forms(orc):
    d, _ = _d(orc, 2, 3)
    C = d.shape[0]
    for A, B in ((250, 1), (400, 3)):
        S, c0 = orc.dense_qubo(d, A, B)
        Sw, c0w = orc.dense_qubo_weighted(d, A, np.full(C - 1, B))
        assert c0 == c0w and np.array_equal(S, Sw)
        rng = np.random.default_rng(A)
        for _ in range(50):
            x = (rng.random(C * C) < 0.3).astype(np.uint8)
            assert orc.energy_terms_weighted(d, A, np.full(C - 1, B), x) == orc.energy_terms(d, A, B, x)[0]


def test_hand_worked_line(orc):
    # a 1x3 line: cells 0, 1, 2 at 0, 100, 200 (scale 100), start 0, leg weights 3 then 1
    d, s = _d(orc, 1, 3)
    assert s == 0 and d[0, 1] == 100 and d[0, 2] == 200
    w = [3, 1]
    assert orc.energy_terms_weighted(d, 500, w, _state([0, 1, 2], 3)) == 3 * 100 + 1 * 100
    assert orc.energy_terms_weighted(d, 500, w, _state([0, 2, 1], 3)) == 3 * 200 + 1 * 100
    # an empty state pays the 2C one-hot penalties
    assert orc.energy_terms_weighted(d, 500, w, np.zeros(9, np.uint8)) == 500 * 6


def test_dense_form_equals_the_terms_on_every_state(orc):
    d, _ = _d(orc, 2, 2)
    C = d.shape[0]
    n = C * C
    w = np.array([7, 3, 2])
    S, c0 = orc.dense_qubo_weighted(d, 900, w)
    assert np.array_equal(S, S.T)
    for bits in range(1 << n):
        x = np.array([(bits >> k) & 1 for k in range(n)], np.uint8)
        assert orc.energy_dense(S, c0, x) == orc.energy_terms_weighted(d, 900, w, x), bits


def test_feasible_minimum_is_the_cheapest_weighted_path(orc):
    d, s = _d(orc, 2, 3, mask=[1, 1, 1, 1, 1, 1])
    C = d.shape[0]
    w = np.array([9, 7, 5, 3, 1])  # a payload that is used up along the path
    A = 2 * int(w.max()) * int(d.max())
    best_state = None
    for rest in itertools.permutations([c for c in range(C) if c != s]):
        path = (s,) + rest
        e = orc.energy_terms_weighted(d, A, w, _state(path, C))
        cost = sum(int(w[t]) * int(d[path[t], path[t + 1]]) for t in range(C - 1))
        assert e == cost
        best_state = e if best_state is None else min(best_state, e)
    # no infeasible state near a path is cheaper: every single flip from the best path costs >= 0
    path = min(((s,) + r for r in itertools.permutations([c for c in range(C) if c != s])),
               key=lambda p: sum(int(w[t]) * int(d[p[t], p[t + 1]]) for t in range(C - 1)))
    x = _state(path, C).reshape(-1)
    e0 = orc.energy_terms_weighted(d, A, w, x)
    assert e0 == best_state
    for k in range(C * C):
        y = x.copy()
        y[k] ^= 1
        assert orc.energy_terms_weighted(d, A, w, y) >= e0


def test_payload_weights_hand_worked():
    from paper_2608_25376_gb300 import objectives
    # 3 cells, dry mass 10, dose 2: legs carry 10 + 2*2 and 10 + 2*1
    assert objectives.payload_leg_weights(3, 10, 2).tolist() == [14, 12]
    w = objectives.payload_leg_weights(5, 7, 3)
    assert w.tolist() == [19, 16, 13, 10] and w.dtype == np.int32
    d = np.array([[0, 100, 200], [100, 0, 100], [200, 100, 0]])
    assert objectives.flight_energy([0, 1, 2], d, [14, 12]) == 14 * 100 + 12 * 100
    assert objectives.within_battery([0, 1, 2], d, [14, 12], 2600) and not objectives.within_battery(
        [0, 2, 1], d, [14, 12], 3999)
    with pytest.raises(ValueError):
        objectives.payload_leg_weights(1, 1, 1)
