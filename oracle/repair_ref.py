"""CPU reference of the path repair -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module.  Plain Python loops over plain lists, one state at a
time, written from the rule the library states for turning a sample into a
flight path (the reconstruction step of Algorithm 1 must hand back a feasible
path; the paper does not say how an infeasible sample becomes one):

* Greedy fix.  Step 0 is the start cell s.  At step t = 1 .. C-1 the
  candidates are the cells not yet on the path whose variable x_{t,i} is 1, or,
  when there is none, every cell not yet on the path; the candidate nearest to
  the previous cell (smallest d, then smallest id) is taken.
* 2-opt on the open path with step 0 fixed.  Move (i, j), 1 <= i < j <= C-1,
  reverses the steps i..j.  One pass takes i = 1 .. C-2 and, for each i,
  j = i+1 .. C-1 in order; a move is applied as soon as it shortens the path,
  and the scan goes on with the next j on the changed path.  Passes repeat while
  the previous one applied a move, at most ``max_passes`` (negative: no limit).

A move is judged here by recomputing the whole path length before and after
the reversal (the library judges it by the two changed edges; both agree
because d is symmetric).  Status: 0 = the state was feasible (every row and
column sum 1 and x_{0,s} = 1) and 2-opt changed nothing, 1 = feasible and
2-opt shortened it, 2 = infeasible.
"""
from __future__ import annotations


def path_length(path, d):
    return sum(int(d[path[t]][path[t + 1]]) for t in range(len(path) - 1))


def is_feasible(x, C, start):
    """x: C*C 0/1 values, t-major (x[t*C + i])."""
    if not x[start]:
        return False
    for t in range(C):
        if sum(1 for i in range(C) if x[t * C + i]) != 1:
            return False
    for i in range(C):
        if sum(1 for t in range(C) if x[t * C + i]) != 1:
            return False
    return True


def greedy_fix(x, d, C, start):
    path = [start]
    used = {start}
    for t in range(1, C):
        prev = path[-1]
        cands = [i for i in range(C) if x[t * C + i] and i not in used]
        if not cands:
            cands = [i for i in range(C) if i not in used]
        nxt = min(cands, key=lambda i: (int(d[prev][i]), i))
        path.append(nxt)
        used.add(nxt)
    return path


def two_opt(path, d, max_passes):
    """-> (path, moved_at_all)"""
    p = list(path)
    C = len(p)
    moved_any = False
    passes = 0
    moved = True
    while moved and (max_passes < 0 or passes < max_passes):
        moved = False
        passes += 1
        for i in range(1, C - 1):
            j = i + 1
            while j <= C - 1:
                q = p[:i] + p[i:j + 1][::-1] + p[j + 1:]
                if path_length(q, d) < path_length(p, d):
                    p = q
                    moved = True
                    moved_any = True
                j += 1
    return p, moved_any


def repair(x, d, C, start, max_passes):
    """-> (path, length, status) for one state x (C*C values, t-major)."""
    x = [int(v) for v in x]
    feasible = is_feasible(x, C, start)
    path = greedy_fix(x, d, C, start)
    path, moved = two_opt(path, d, max_passes) if max_passes != 0 else (path, False)
    status = 2 if not feasible else (1 if moved else 0)
    return path, path_length(path, d), status
