"""The extended objective: flight energy under a payload that is sprayed away.

Section V of the paper names battery capacity and the pesticide application
amount as the objectives to add next and gives no formula.  The reading here
keeps the QUBO quadratic: the UAV sprays the same dose on every cell, so the
mass it carries on the leg from step t to step t+1 is dry + dose * (C - 1 - t)
(the start cell is sprayed at step 0), and a leg's flight energy is taken as
proportional to mass times distance.  The per-leg weights go to
qp_build_qubo_weighted; the battery is a budget on the resulting energy,
checked on the path found (an inequality inside the QUBO would need slack
variables).
"""
from __future__ import annotations

import numpy as np


def payload_leg_weights(C: int, dry: int, dose: int) -> np.ndarray:
    """w_t = dry + dose * (C - 1 - t) for t = 0 .. C-2 (integer mass units)."""
    if C < 2 or dry < 0 or dose < 0:
        raise ValueError("need C >= 2, dry >= 0 and dose >= 0")
    t = np.arange(C - 1, dtype=np.int64)
    w = dry + dose * (C - 1 - t)
    if w.max(initial=0) > np.iinfo(np.int32).max:
        raise ValueError("leg weights beyond int32")
    return w.astype(np.int32)


def flight_energy(path, d, w) -> int:
    """sum_t w_t d(path_t, path_t+1): the weighted distance term of a path."""
    d = np.asarray(d)
    return int(sum(int(w[t]) * int(d[path[t], path[t + 1]]) for t in range(len(path) - 1)))


def within_battery(path, d, w, capacity) -> bool:
    """Whether the path's flight energy fits the battery budget (same units)."""
    return flight_energy(path, d, w) <= capacity
