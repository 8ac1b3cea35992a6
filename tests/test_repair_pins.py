"""Pins of the repair reference (oracle/repair_ref.py) against hand-worked
cases, closed forms and exhaustive checks -- no GPU.

The rule being pinned: greedy fix (hot cells of the row first, nearest to the
previous cell, ties to the smaller id), then first-improvement 2-opt passes on
the open path with the start fixed."""
import itertools
import random

import numpy as np
import pytest

from oracle import repair_ref as rr


def strip(L):
    """A 1 x L row of cells at unit pitch, scale 100: d = 100 |i - j| exactly."""
    return [[100 * abs(i - j) for j in range(L)] for i in range(L)]


def grid_d(rows, cols):
    """Full rows x cols grid, d = round(100 * euclid) by integer square root."""
    import math
    cells = [(r, c) for r in range(rows) for c in range(cols)]
    d = []
    for (r1, c1) in cells:
        row = []
        for (r2, c2) in cells:
            N = 10000 * ((r1 - r2) ** 2 + (c1 - c2) ** 2)
            s = math.isqrt(N)
            row.append(s + (1 if N - s * s > s else 0))
        d.append(row)
    return d


def state_of(rows_hot, C):
    """rows_hot[t] = cells hot in row t -> flat t-major 0/1 list."""
    x = [0] * (C * C)
    for t, hot in enumerate(rows_hot):
        for i in hot:
            x[t * C + i] = 1
    return x


def test_hand_case_duplicate_and_empty_row():
    # 1x4 strip from cell 0.  Row 2 repeats cell 2, row 3 is empty.
    d = strip(4)
    x = state_of([[0], [2], [2], []], 4)
    # t=1: hot {2}.  t=2: 2 is taken, no hot candidate -> unused {1, 3}, both
    # 100 from cell 2 -> smaller id 1.  t=3: only 3 is left.
    assert rr.repair(x, d, 4, 0, 0) == ([0, 2, 1, 3], 500, 2)
    # 2-opt: move (1, 2) turns 0-2-1-3 into 0-1-2-3 (400 -> 200 on the two
    # changed edges); nothing shortens 0-1-2-3.
    assert rr.repair(x, d, 4, 0, -1) == ([0, 1, 2, 3], 300, 2)


def test_hand_case_two_hot_cells_nearest_wins():
    d = strip(5)
    x = state_of([[0], [1, 4], [4], [], []], 5)
    # t=1: hot {1, 4} -> 1 (100 < 400).  t=2: hot {4}.  t=3: no hot -> unused
    # {2, 3} from 4 -> 3.  t=4: 2.
    assert rr.repair(x, d, 5, 0, 0) == ([0, 1, 4, 3, 2], 600, 2)


def test_feasible_state_is_its_own_path():
    rnd = random.Random(5)
    d = grid_d(3, 4)
    C = 12
    for _ in range(20):
        perm = [0] + rnd.sample(range(1, C), C - 1)
        x = state_of([[c] for c in perm], C)
        path, L, status = rr.repair(x, d, C, 0, 0)
        assert path == perm and status == 0
        assert L == sum(d[perm[t]][perm[t + 1]] for t in range(C - 1))


def test_start_not_hot_makes_the_state_infeasible():
    d = strip(3)
    x = state_of([[1], [0], [2]], 3)  # a permutation, but step 0 is not the start
    path, L, status = rr.repair(x, d, 3, 0, 0)
    assert status == 2 and path[0] == 0 and sorted(path) == [0, 1, 2]


def no_improving_move(path, d):
    """Exhaustive: no reversal of steps i..j (1 <= i < j <= C-1) is shorter."""
    L0 = rr.path_length(path, d)
    C = len(path)
    for i in range(1, C - 1):
        for j in range(i + 1, C):
            q = path[:i] + path[i:j + 1][::-1] + path[j + 1:]
            if rr.path_length(q, d) < L0:
                return False
    return True


@pytest.mark.parametrize("rows,cols,start", [(1, 6, 0), (3, 3, 4), (3, 4, 0), (4, 4, 5), (2, 5, 9)])
def test_random_states_give_2opt_local_optima(rows, cols, start):
    rnd = random.Random(rows * 100 + cols)
    d = grid_d(rows, cols)
    C = rows * cols
    for _ in range(8):
        x = [1 if rnd.random() < 1.5 / C else 0 for _ in range(C * C)]
        p0, L0, _ = rr.repair(x, d, C, start, 0)
        p, L, status = rr.repair(x, d, C, start, -1)
        assert sorted(p) == list(range(C)) and p[0] == start
        assert sorted(p0) == list(range(C)) and p0[0] == start
        assert L <= L0 and L == rr.path_length(p, d)
        assert no_improving_move(p, d)
        assert L >= 100 * (C - 1)  # every step joins two cells at least one pitch apart


def test_passes_compose():
    """Two passes from scratch == one pass applied twice (each pass starts from
    the previous one's path)."""
    rnd = random.Random(11)
    d = grid_d(4, 5)
    C = 20
    for _ in range(6):
        perm = [0] + rnd.sample(range(1, C), C - 1)
        one, _ = rr.two_opt(perm, d, 1)
        twice, _ = rr.two_opt(one, d, 1)
        two, _ = rr.two_opt(perm, d, 2)
        assert twice == two


@pytest.mark.parametrize("rows,cols", [(3, 3), (3, 4), (4, 5), (6, 6)])
def test_serpentine_is_kept(rows, cols):
    """Closed form: a serpentine from the corner is optimal (100 (C-1)), so
    2-opt leaves it alone and the status is 0."""
    C = rows * cols
    order = []
    for r in range(rows):
        cs = range(cols) if r % 2 == 0 else range(cols - 1, -1, -1)
        order += [r * cols + c for c in cs]
    x = state_of([[c] for c in order], C)
    path, L, status = rr.repair(x, grid_d(rows, cols), C, 0, -1)
    assert path == order and L == 100 * (C - 1) and status == 0


def test_two_opt_at_least_brute_force_optimum_tiny():
    rnd = random.Random(3)
    d = grid_d(2, 3)
    C = 6
    best = min(rr.path_length([0] + list(p), d) for p in itertools.permutations(range(1, C)))
    assert best == 500
    for _ in range(10):
        x = [1 if rnd.random() < 0.3 else 0 for _ in range(C * C)]
        _, L, _ = rr.repair(x, d, C, 0, -1)
        assert L >= best


def test_degenerate_sizes():
    assert rr.repair([1], [[0]], 1, 0, -1) == ([0], 0, 0)
    assert rr.repair([0], [[0]], 1, 0, -1) == ([0], 0, 2)
    d = strip(2)
    assert rr.repair(state_of([[0], [1]], 2), d, 2, 0, -1) == ([0, 1], 100, 0)
    assert rr.repair([0, 0, 0, 0], d, 2, 0, -1) == ([0, 1], 100, 2)
