"""GPU parity of the path repair (greedy fix + 2-opt) and of the time-budgeted
anneal, through the C ABI, against the CPU references.

Repair: paths, lengths and statuses are integers and must match the reference
exactly for every state (small cases) or for sampled states (large batches,
where every state is independent), with properties checked on the rest.
Timed mode: the call is reproduced from the sweeps and rounds it reports --
the oracle anneals each round's replicas, the repair reference repairs them,
and the shortest path (ties to the smaller replica) must be the one returned.
"""
import numpy as np
import pytest

from conftest import has_gpu
from oracle import repair_ref as rr
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs
from paper_2608_25376_gb300 import qpath

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import torch
    qbuild.build()
    qpath.lib()
    return torch.device("cuda:0")


def problem(orc, f):
    return orc.Problem(f.rows, f.cols, f.free_mask, f.start)


def mixed_states(C, count, seed, s):
    """Feasible permutations, Bernoulli(1/C) and Bernoulli(2.5/C) states, an
    all-zero and an all-one state, in turn."""
    rng = np.random.Generator(np.random.PCG64(seed))
    X = np.zeros((count, C * C), np.uint8)
    for r in range(count):
        k = r % 5
        if k == 0:
            perm = np.concatenate([[s], rng.permutation(np.setdiff1d(np.arange(C), [s]))])
            X[r].reshape(C, C)[np.arange(C), perm] = 1
        elif k == 1:
            X[r] = rng.random(C * C) < 1.0 / C
        elif k == 2:
            X[r] = rng.random(C * C) < 2.5 / C
        elif k == 3:
            X[r] = 0
        else:
            X[r] = 1
    return X


def gpu_repair(h, X, passes, host=False):
    import torch
    R = X.shape[0]
    C = h.info["C"]
    if host:
        P = np.zeros((R, C), np.int32)
        L = np.zeros(R, np.int64)
        S = np.zeros(R, np.int32)
        qpath.qp_repair_batch(h, R, np.ascontiguousarray(X), passes, P, L, S)
        return P, L, S
    Xd = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    P = torch.zeros((R, C), dtype=torch.int32, device="cuda")
    L = torch.zeros(R, dtype=torch.int64, device="cuda")
    S = torch.zeros(R, dtype=torch.int32, device="cuda")
    qpath.qp_repair_batch(h, R, Xd, passes, P, L, S, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return P.cpu().numpy(), L.cpu().numpy(), S.cpu().numpy()


def check_against_reference(P, L, S, X, d, C, s, passes, rows):
    dl = d.tolist()
    for r in rows:
        path, length, status = rr.repair(X[r].tolist(), dl, C, s, passes)
        assert P[r].tolist() == path, (r, P[r][:12], path[:12])
        assert L[r] == length and S[r] == status, (r, L[r], length, S[r], status)


def check_properties(P, L, S, d, C, s):
    assert (P[:, 0] == s).all()
    assert (np.sort(P, axis=1) == np.arange(C)).all()
    assert (L == d[P[:, :-1], P[:, 1:]].sum(axis=1)).all()
    assert np.isin(S, [0, 1, 2]).all()


CASES = [
    ("1x2", inputs.rect(1, 2)),
    ("1x5", inputs.rect(1, 5)),
    ("3x4", inputs.rect(3, 4)),
    ("3x5-start7", inputs.rect(3, 5, start=7)),
    ("6x6-p0.2", inputs.obstacles(6, 6, 0.2, seed=3, start=14)),
    ("7x7", inputs.rect(7, 7, start=24)),
]


@pytest.mark.parametrize("passes", [0, 1, -1])
@pytest.mark.parametrize("name,f", CASES)
def test_repair_parity_small(dev, orc, name, f, passes):
    Pr = problem(orc, f)
    C, s = Pr.C, Pr.start_cell
    h = qpath.qp_build_qubo(f)
    X = mixed_states(C, 37, seed=C * 7 + passes, s=s)  # 37: several CTAs and a ragged tail
    P, L, S = gpu_repair(h, X, passes)
    check_properties(P, L, S, Pr.d, C, s)
    check_against_reference(P, L, S, X, Pr.d, C, s, passes, range(37))
    # host buffers take the staged, synchronous route to the same result
    P2, L2, S2 = gpu_repair(h, X, passes, host=True)
    assert (P2 == P).all() and (L2 == L).all() and (S2 == S).all()


def test_repair_of_annealed_states(dev, orc):
    """States the oracle's sampler ends in (mostly one-hot, some broken)."""
    f = inputs.obstacles(6, 6, 0.15, seed=2)
    Pr = problem(orc, f)
    ref = orc.anneal_structured(Pr, 24, 40, seed=5)
    h = qpath.qp_build_qubo(f)
    for passes in (0, -1):
        P, L, S = gpu_repair(h, ref.states, passes)
        check_against_reference(P, L, S, ref.states, Pr.d, Pr.C, Pr.start_cell, passes, range(24))
    # a feasible final state comes out as its decoded path when 2-opt is off
    P, L, S = gpu_repair(h, ref.states, 0)
    for r in range(24):
        dec = qpath.qp_decode_path(h, ref.states[r])
        if dec is not None:
            assert S[r] == 0 and (P[r] == dec[0]).all() and L[r] == dec[1]
        else:
            assert S[r] == 2


def test_repair_full_size_10x10_sampled(dev, orc):
    """1024 states of the 10x10 obstacle field (92 cells), as the benchmark's
    batch; sampled states against the reference, properties on all."""
    f = inputs.WORKLOADS["10x10-p0.10"]["field"]()
    Pr = problem(orc, f)
    C, s = Pr.C, Pr.start_cell
    h = qpath.qp_build_qubo(f)
    X = mixed_states(C, 1024, seed=17, s=s)
    P, L, S = gpu_repair(h, X, -1)
    check_properties(P, L, S, Pr.d, C, s)
    check_against_reference(P, L, S, X, Pr.d, C, s, -1, [0, 1, 2, 3, 4, 511, 1023])
    # every result is a 2-opt local optimum: no reversal (i, j) shortens it
    D = Pr.d.astype(np.int64)
    for r in range(0, 1024, 97):
        p = P[r]
        for i in range(1, C - 1):
            j = np.arange(i + 1, C)
            old = D[p[i - 1], p[i]] + np.where(j + 1 < C, D[p[j], p[np.minimum(j + 1, C - 1)]], 0)
            new = D[p[i - 1], p[j]] + np.where(j + 1 < C, D[p[i], p[np.minimum(j + 1, C - 1)]], 0)
            assert (new >= old).all(), (r, i)


def test_repair_large_field_greedy(dev, orc):
    """A field near the 512-cell mark: the greedy fix against the reference,
    2-opt (one pass) by its properties."""
    f = inputs.obstacles(24, 24, 0.15, seed=1)
    Pr = problem(orc, f)
    C, s = Pr.C, Pr.start_cell
    h = qpath.qp_build_qubo(f)
    X = mixed_states(C, 9, seed=23, s=s)
    P, L, S = gpu_repair(h, X, 0)
    check_properties(P, L, S, Pr.d, C, s)
    check_against_reference(P, L, S, X, Pr.d, C, s, 0, range(9))
    P1, L1, S1 = gpu_repair(h, X, 1)
    check_properties(P1, L1, S1, Pr.d, C, s)
    assert (L1 <= L).all()


def test_repair_at_1024_cells(dev, orc):
    """A 32 x 32 field (1024 cells; 8.3 KB of path, edge and used-cell buffers
    per warp): the greedy fix against the reference on sampled states, one
    2-opt pass by its properties on all of them."""
    f = inputs.rect(32, 32, start=527)
    Pr = problem(orc, f)
    C, s = Pr.C, Pr.start_cell
    assert C == 1024
    h = qpath.qp_build_qubo(f)
    X = mixed_states(C, 6, seed=41, s=s)
    P, L, S = gpu_repair(h, X, 0)
    check_properties(P, L, S, Pr.d, C, s)
    check_against_reference(P, L, S, X, Pr.d, C, s, 0, [0, 1, 3])
    P1, L1, S1 = gpu_repair(h, X, 1)
    check_properties(P1, L1, S1, Pr.d, C, s)
    assert (L1 <= L).all()


def test_repair_rejects_generic_qubo(dev):
    S = np.zeros((4, 4), np.int32)
    h = qpath.qp_build_from_dense(S)
    with pytest.raises(qpath.QpError):
        qpath.qp_repair_path(h, np.zeros(4, np.uint8))


# ----------------------------------------------------------------- time-budgeted anneal
def reproduce_timed(orc, Pr, R, out, T0, T1, seed, passes):
    """The oracle's version of a timed call with the sweeps and rounds it reported."""
    n_sw, rounds = out["n_sweeps"], out["rounds"]
    best = None
    dl = Pr.d.tolist()
    feasible = 0
    for k in range(rounds):
        idx = np.arange(k * R, (k + 1) * R, dtype=np.int32)
        ref = orc.anneal_structured(Pr, idx, n_sw, T0=T0, T1=T1, seed=seed)
        for r in range(R):
            path, length, status = rr.repair(ref.states[r].tolist(), dl, Pr.C, Pr.start_cell, passes)
            feasible += status != 2
            if best is None or length < best[0]:
                best = (length, k * R + r, path, status, int(ref.energies[r]), ref.states[r])
    return best, feasible


@pytest.mark.parametrize("passes", [0, -1])
def test_timed_reproducible_from_its_report(dev, orc, passes):
    f = inputs.rect(4, 4)
    Pr = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    R, T0, T1, seed = 32, 1e3, 1.0, 9
    sc = qpath.schedule(120, T0, T1)
    out = qpath.qp_anneal_timed(h, R, sc, seed, time_limit_ms=15.0, max_passes=passes, want_state=True)
    assert out["n_sweeps"] >= 1 and out["rounds"] >= 1
    assert out["rounds"] * R * out["n_sweeps"] * (Pr.C - 1) ** 2 < 4e8, "budget too generous for the oracle"
    best, feasible = reproduce_timed(orc, Pr, R, out, T0, T1, seed, passes)
    length, replica, path, status, energy, state = best
    assert out["length"] == length and out["replica"] == replica
    assert out["path"].tolist() == path and out["status"] == status and out["energy"] == energy
    assert (out["state"] == state).all()
    assert out["n_feasible"] == feasible
    assert out["elapsed_ms"] >= out["probe_ms"] > 0


def test_timed_fits_a_long_schedule_to_the_budget(dev, orc):
    """A schedule far too long for the budget is replaced by a shorter one of
    m * 2^e sweeps; the result is that schedule's single round."""
    f = inputs.obstacles(10, 10, 0.10, seed=1)
    Pr = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    R, seed = 256, 4
    sc = qpath.schedule(4000, 1e3, 1.0)
    out = qpath.qp_anneal_timed(h, R, sc, seed, time_limit_ms=8.0, max_passes=0)
    n = out["n_sweeps"]
    assert 1 <= n < 4000
    if n >= 16:
        e = int(np.floor(np.log2(n))) - 3
        assert n % (1 << e) == 0 and 8 <= n >> e < 16
    # the returned replica's path is the repaired final state of that schedule
    r = out["replica"]
    k = r // R
    ref = orc.anneal_structured(Pr, np.array([r], np.int32), n, seed=seed)
    path, length, status = rr.repair(ref.states[0].tolist(), Pr.d.tolist(), Pr.C, Pr.start_cell, 0)
    assert out["path"].tolist() == path and out["length"] == length and out["status"] == status
    assert k < out["rounds"]


@pytest.mark.parametrize("rows,cols", inputs.PAPER_GRIDS)
def test_timed_paper_grids(dev, rows, cols):
    """The paper's protocol (Section IV-C): full grids from a corner with a
    100 ms limit.  No path is shorter than 100 (C-1) (every step joins two
    cells at least one pitch apart); 3x3 must reach it."""
    f = inputs.rect(rows, cols)
    h = qpath.qp_build_qubo(f)
    out = qpath.qp_anneal_timed(h, 1024, qpath.schedule(2000), 1, time_limit_ms=100.0, max_passes=0)
    C = rows * cols
    assert sorted(out["path"].tolist()) == list(range(C)) and out["path"][0] == 0
    assert out["length"] >= 100 * (C - 1)
    if C == 9:
        assert out["length"] == 800
    assert out["rounds"] >= 1 and out["n_feasible"] >= 1
