"""Seeded synthetic fields shaped like the paper's workloads.

This module only draws inputs: grid sizes, obstacle masks, irregular boundary
masks and start cells.  It holds none of the method's arithmetic (no distances,
no QUBO, no annealing) and is the one module that both the CUDA path's tests and
the oracle's tests take their inputs from.

Recipes (the paper uses full M x N grids of 3x3 ... 6x6 cells, Section IV-C,
Table II; it names no dataset):
  * ``rect``      -- obstacle-free M x N grid, start at grid cell 0.
  * ``obstacles`` -- M x N grid, each cell an obstacle with probability p
                     (independent draws from numpy's PCG64 seeded with ``seed``);
                     the start cell is forced free.
  * ``fields_8_16`` -- rectangles with sides in [8, 16] (or fixed squares) and
                     obstacle probability uniform in [0, 0.2]; start = first
                     free cell.  Training seeds and held-out seeds are disjoint.
  * ``batch``     -- ``count`` fields with sides H, W uniform in [lo, hi],
                     obstacle probability uniform in [0, p_max], and an
                     irregular boundary: each row loses 0..floor(W/4) cells at
                     each end.  The start is the first free cell in row-major
                     order.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Field:
    rows: int
    cols: int
    free_mask: np.ndarray  # uint8 [rows*cols], 1 = a cell to visit
    start: int             # grid index r*cols + c of the start cell (free)

    @property
    def n_cells(self) -> int:
        return int(self.free_mask.sum())


def rect(rows: int, cols: int, start: int = 0) -> Field:
    return Field(rows, cols, np.ones(rows * cols, np.uint8), start)


def obstacles(rows: int, cols: int, p: float, seed: int, start: int = 0) -> Field:
    rng = np.random.Generator(np.random.PCG64(seed))
    mask = (rng.random(rows * cols) >= p).astype(np.uint8)
    mask[start] = 1
    return Field(rows, cols, mask, start)


def batch(count: int, seed: int, lo: int = 4, hi: int = 16, p_max: float = 0.2) -> list[Field]:
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        H = int(rng.integers(lo, hi + 1))
        W = int(rng.integers(lo, hi + 1))
        p = float(rng.uniform(0.0, p_max))
        mask = (rng.random(H * W) >= p).astype(np.uint8).reshape(H, W)
        trim = W // 4
        for r in range(H):
            a = int(rng.integers(0, trim + 1))
            b = int(rng.integers(0, trim + 1))
            if a:
                mask[r, :a] = 0
            if b:
                mask[r, W - b:] = 0
        flat = mask.reshape(-1)
        free = np.flatnonzero(flat)
        if free.size < 2:  # keep every field a real path problem
            flat[:2] = 1
            free = np.flatnonzero(flat)
        out.append(Field(H, W, flat.astype(np.uint8), int(free[0])))
    return out


def fields_8_16(count: int, seed: int, lo: int = 8, hi: int = 16, p_max: float = 0.2,
                square: int = 0) -> list[Field]:
    """Rectangles with sides uniform in [lo, hi] (or square x square when
    square > 0) and obstacle probability uniform in [0, p_max]; the start is the
    first free cell in row-major order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for _ in range(count):
        H = square or int(rng.integers(lo, hi + 1))
        W = square or int(rng.integers(lo, hi + 1))
        p = float(rng.uniform(0.0, p_max))
        mask = (rng.random(H * W) >= p).astype(np.uint8)
        free = np.flatnonzero(mask)
        if free.size < 2:
            mask[:2] = 1
            free = np.flatnonzero(mask)
        out.append(Field(H, W, mask, int(free[0])))
    return out


# The paper's grid sweep (Section IV-C, Table II) and the workloads the
# throughput metric is quoted on.
PAPER_GRIDS = [(3, 3), (3, 4), (4, 4), (4, 5), (5, 5), (5, 6), (6, 6)]

WORKLOADS = {
    "4x4-dense": dict(field=lambda: rect(4, 4), replicas=64, n_sweeps=2000, seed=1, kernel="dense"),
    "10x10-p0.10": dict(field=lambda: obstacles(10, 10, 0.10, seed=1), replicas=1024, n_sweeps=5000,
                        seed=1, kernel="structured"),
    "24x24-p0.15": dict(field=lambda: obstacles(24, 24, 0.15, seed=1), replicas=4096, n_sweeps=10000,
                        seed=1, kernel="structured"),
}
T0_DEFAULT = 1e3
T1_DEFAULT = 1.0
