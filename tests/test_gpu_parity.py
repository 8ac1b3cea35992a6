"""GPU parity: the CUDA sweeps through the C ABI against the CPU oracle.

The bar is bit-exactness: final states, final int64 energies, best feasible
energies and accepted-flip counts per replica, for the same seed.  Small
cases run every replica; the full-size workloads (in the launch
configuration the benchmark times) compare sampled replicas, which is exact
because every replica's random stream is fixed by its global index.
"""
import ctypes as ct

import numpy as np
import pytest

from conftest import has_gpu
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


def gpu_anneal(h, R, n_sweeps, seed, T0=1e3, T1=1.0, sweep_begin=0, sweep_end=None, init=None,
               kernel=qpath.QP_KERNEL_AUTO, rpc=0, offset=0, host=False):
    import torch
    n = h.info["n"]
    sc = qpath.schedule(n_sweeps, T0, T1, sweep_begin, sweep_end)
    if host:
        st = np.zeros((R, n), np.uint8)
        E = np.zeros(R, np.int64)
        B = np.zeros(R, np.int64)
        A = np.zeros(R, np.int64)
        qpath.qp_anneal_ex(h, R, sc, seed, init, st, E, B, kernel=kernel, replicas_per_cta=rpc,
                           replica_offset=offset, accepts_out=A)
        return st, E, B, A
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    A = torch.zeros(R, dtype=torch.int64, device="cuda")
    ini = None if init is None else torch.from_numpy(np.ascontiguousarray(init)).cuda()
    qpath.qp_anneal_ex(h, R, sc, seed, ini, st, E, B, kernel=kernel, replicas_per_cta=rpc,
                       replica_offset=offset, accepts_out=A, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy(), A.cpu().numpy()


def problem(orc, f, A=None, B=1):
    return orc.Problem(f.rows, f.cols, f.free_mask, f.start, A=A, B=B)


def assert_same(got, ref, idx=None):
    st, E, B, A = got
    if idx is not None:
        st, E, B, A = st[idx], E[idx], B[idx], A[idx]
    assert (E == ref.energies).all(), (E[:8], ref.energies[:8])
    assert (B == ref.best).all()
    assert (A == ref.accepts).all()
    assert (st == ref.states).all()


FIELDS = [
    ("1x2", inputs.rect(1, 2)),
    ("3x3", inputs.rect(3, 3)),
    ("4x4", inputs.rect(4, 4)),
    ("3x5-start7", inputs.rect(3, 5, start=7)),
    ("6x6-p0.2", inputs.obstacles(6, 6, 0.2, seed=3, start=14)),
    ("10x10-p0.1", inputs.obstacles(10, 10, 0.1, seed=1)),
    ("13x13-p0.1", inputs.obstacles(13, 13, 0.1, seed=5, start=20)),
]


# ----------------------------------------------------------------- build
@pytest.mark.parametrize("name,f", FIELDS[1:6])
def test_build_matches_oracle(dev, orc, name, f):
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f, flags=qpath.QP_STRUCTURED | qpath.QP_DENSE)
    info = h.info
    assert info["C"] == P.C and info["n"] == P.n and info["max_d"] == P.max_d and info["A"] == P.A
    assert (qpath.qp_export_dist(h) == P.d).all()
    S, c0 = P.dense()
    assert info["c0"] == c0
    assert (qpath.qp_export_dense(h) == S).all()


# ----------------------------------------------------------------- structured sweep
STRUCT_KERNELS = [("rows", qpath.QP_KERNEL_STRUCTURED_ROWS), ("flat", qpath.QP_KERNEL_STRUCTURED_FLAT),
                  ("group", qpath.QP_KERNEL_STRUCTURED_GROUP)]


def kernel_fits(kernel, C):
    if kernel == qpath.QP_KERNEL_STRUCTURED_GROUP:
        return C <= 128
    if kernel == qpath.QP_KERNEL_STRUCTURED_ROWS:
        return C <= 512
    return True


@pytest.mark.parametrize("kname,kernel", STRUCT_KERNELS)
@pytest.mark.parametrize("name,f", FIELDS)
def test_structured_parity(dev, orc, name, f, kname, kernel):
    P = problem(orc, f)
    if not kernel_fits(kernel, P.C):
        pytest.skip("field too large for this kernel")
    R, S = (32, 300) if P.C <= 40 else (8, 60)
    h = qpath.qp_build_qubo(f)
    ref = orc.anneal_structured(P, R, S, seed=7)
    assert_same(gpu_anneal(h, R, S, 7, kernel=kernel), ref)


@pytest.mark.parametrize("kname,kernel", STRUCT_KERNELS)
def test_structured_multichunk(dev, orc, kname, kernel):
    """256 < C <= 512: rows span several 128-wide chunks with a ragged tail (the
    row kernel's widest variant); the flat kernel keeps its spins in global
    memory here."""
    f = inputs.obstacles(18, 18, 0.1, seed=8, start=5)
    P = problem(orc, f)
    if not kernel_fits(kernel, P.C):
        pytest.skip("field too large for this kernel")
    assert 256 < P.C <= 512
    h = qpath.qp_build_qubo(f)
    ref = orc.anneal_structured(P, 3, 12, seed=3)
    assert_same(gpu_anneal(h, 3, 12, 3, kernel=kernel), ref)


@pytest.mark.parametrize("kname,kernel", STRUCT_KERNELS)
@pytest.mark.parametrize("rows,cols", [(8, 16), (3, 43), (16, 16), (1, 257)])
def test_structured_at_chunk_boundaries(dev, orc, rows, cols, kname, kernel):
    """C = 128, 129, 256, 257: the last field of one 128-column chunk per lane
    and the first of two, the last of two and the first of four (here a single
    257-cell row of the grid, so every step is along one line)."""
    f = inputs.rect(rows, cols)
    P = problem(orc, f)
    assert P.C == rows * cols
    if not kernel_fits(kernel, P.C):
        pytest.skip("field too large for this kernel")
    h = qpath.qp_build_qubo(f)
    R, S = (6, 8) if P.C <= 128 else (4, 5)
    ref = orc.anneal_structured(P, R, S, seed=9)
    assert_same(gpu_anneal(h, R, S, 9, kernel=kernel), ref)


def test_structured_above_512_cells_falls_back(dev, orc):
    f = inputs.obstacles(24, 24, 0.05, seed=8)
    P = problem(orc, f)
    assert P.C > 512
    h = qpath.qp_build_qubo(f)
    ref = orc.anneal_structured(P, 2, 3, seed=3)
    assert_same(gpu_anneal(h, 2, 3, 3), ref)


@pytest.mark.parametrize("rows,cols,kernel", [(16, 32, qpath.QP_KERNEL_STRUCTURED_ROWS),
                                              (16, 32, qpath.QP_KERNEL_STRUCTURED_FLAT),
                                              (17, 31, qpath.QP_KERNEL_STRUCTURED)])
def test_structured_at_the_row_kernel_limit(dev, orc, rows, cols, kernel):
    """C = 512 (the row kernel's widest field: four 128-column chunks per lane,
    no ragged tail) with both kernels, and C = 527 just past it (the automatic
    choice falls back to the flat kernel)."""
    f = inputs.rect(rows, cols, start=rows * cols - 1)
    P = problem(orc, f)
    assert P.C == rows * cols
    h = qpath.qp_build_qubo(f)
    ref = orc.anneal_structured(P, 3, 4, seed=12, T0=3000.0, T1=2000.0)
    assert_same(gpu_anneal(h, 3, 4, 12, T0=3000.0, T1=2000.0, kernel=kernel), ref)


@pytest.mark.slow
def test_structured_at_the_cell_limit(dev, orc):
    """C = 4096, the library's largest field (64 x 64, n = 16.8M variables per
    replica, spins in global memory): one replica (index 1 of 2), one sweep."""
    f = inputs.rect(64, 64, start=2080)
    P = problem(orc, f)
    assert P.C == 4096
    h = qpath.qp_build_qubo(f)
    ref = orc.anneal_structured(P, [1], 1, seed=5, T0=2000.0, T1=2000.0)
    got = gpu_anneal(h, 2, 1, 5, T0=2000.0, T1=2000.0)
    assert_same(got, ref, [1])
    with pytest.raises(qpath.QpError):
        qpath.qp_build_qubo(inputs.rect(64, 65))  # one cell more than the limit


@pytest.mark.parametrize("kname,kernel", STRUCT_KERNELS)
@pytest.mark.parametrize("rpc", [1, 2, 3, 8, 16])
def test_structured_replicas_per_cta(dev, orc, rpc, kname, kernel):
    f = inputs.obstacles(7, 7, 0.15, seed=2)
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    ref = orc.anneal_structured(P, 21, 80, seed=11)
    assert_same(gpu_anneal(h, 21, 80, 11, rpc=rpc, kernel=kernel), ref)


@pytest.mark.parametrize("kname,kernel", STRUCT_KERNELS)
def test_structured_hot_start(dev, orc, kname, kernel):
    """Dense random initial states (many hot cells per row) at a high fixed
    temperature: every draw path, many accepts per row."""
    f = inputs.obstacles(9, 11, 0.1, seed=12, start=3)
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    rng = np.random.default_rng(12)
    R = 10
    init = (rng.random((R, P.n)) < 0.4).astype(np.uint8)
    ref = orc.anneal_structured(P, R, 30, seed=13, init_states=init, T0=5e4, T1=5e4)
    assert_same(gpu_anneal(h, R, 30, 13, T0=5e4, T1=5e4, init=init, kernel=kernel), ref)


@pytest.mark.parametrize("T0,T1", [(24000.0, 20000.0), (26000.0, 25000.0), (1500.0, 900.0), (40.0, 3.0),
                                   (2.0, 0.25)])
@pytest.mark.parametrize("kname,kernel", STRUCT_KERNELS)
def test_structured_temperature_edges(dev, orc, kname, kernel, T0, T1):
    """Schedules around the row kernel's switch between acceptance bounds
    (T below ~24500) and per-pass table tests (above), and very cold ones:
    dense random starts give many accepts and many draws per row."""
    f = inputs.obstacles(8, 9, 0.1, seed=21, start=5)
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    rng = np.random.default_rng(int(T0))
    R = 12
    init = (rng.random((R, P.n)) < 0.3).astype(np.uint8)
    ref = orc.anneal_structured(P, R, 25, seed=17, init_states=init, T0=T0, T1=T1)
    assert_same(gpu_anneal(h, R, 25, 17, T0=T0, T1=T1, init=init, kernel=kernel), ref)


@pytest.mark.parametrize("kname,kernel", STRUCT_KERNELS)
def test_structured_int32_distances(dev, orc, kname, kernel):  # 23 cells: every kernel fits
    """scale = 10000 forces int32 distances while the dE bound still fits."""
    f = inputs.obstacles(5, 5, 0.1, seed=4)
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start, scale=10000)
    assert P.max_d > 32767
    h = qpath.qp_build_qubo(f, scale=10000)
    ref = orc.anneal_structured(P, 16, 100, seed=2)
    assert_same(gpu_anneal(h, 16, 100, 2, kernel=kernel), ref)


def test_init_states_offset_seed_and_host_buffers(dev, orc):
    f = inputs.obstacles(8, 8, 0.1, seed=6)
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    rng = np.random.default_rng(0)
    R = 12
    init = (rng.random((R, P.n)) < 0.05).astype(np.uint8)
    seed = 0xDEADBEEF12345678
    ref = orc.anneal_structured(P, list(range(100, 100 + R)), 150, seed=seed, init_states=init,
                                T0=200.0, T1=2.0)
    got = gpu_anneal(h, R, 150, seed, T0=200.0, T1=2.0, init=init, offset=100, host=True)
    assert_same(got, ref)


def test_resume_equals_one_run(dev, orc):
    f = inputs.obstacles(9, 9, 0.1, seed=9)
    h = qpath.qp_build_qubo(f)
    S = 400
    full = gpu_anneal(h, 16, S, 5)
    a = gpu_anneal(h, 16, S, 5, sweep_end=150)
    b = gpu_anneal(h, 16, S, 5, sweep_begin=150, init=a[0])
    assert (full[0] == b[0]).all() and (full[1] == b[1]).all()
    assert (full[2] == np.minimum(a[2], b[2])).all()


def test_zero_sweeps_and_single_sweep(dev, orc):
    f = inputs.obstacles(5, 5, 0.1, seed=1)
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    st, E, B, A = gpu_anneal(h, 4, 10, 1, sweep_begin=4, sweep_end=4)
    x0 = np.zeros((P.C, P.C), np.uint8)
    x0[0, P.start_cell] = 1
    assert (st == x0.reshape(-1)).all() and (E == P.energy(x0)).all()
    assert (B == qpath.E_NONE).all() and (A == 0).all()
    ref = orc.anneal_structured(P, 4, 1, seed=1, T0=30.0, T1=30.0)
    assert_same(gpu_anneal(h, 4, 1, 1, T0=30.0, T1=30.0), ref)


# ----------------------------------------------------------------- dense sweep
def test_dense_path_parity_4x4_full_workload(dev, orc):
    """4x4 obstacle-free grid, dense int32 Q, 64 replicas x 2000 sweeps, seed 1:
    the whole workload, every replica."""
    f = inputs.rect(4, 4)
    P = problem(orc, f)
    S, c0 = P.dense()
    fr, fv = P.frozen()
    h = qpath.qp_build_qubo(f, flags=qpath.QP_DENSE)
    ref = orc.anneal_dense(S, c0, 64, 2000, seed=1, frozen=fr, frozen_val=fv, C=P.C)
    assert_same(gpu_anneal(h, 64, 2000, 1, kernel=qpath.QP_KERNEL_DENSE), ref)


@pytest.mark.parametrize("name,f", FIELDS[1:6])
def test_dense_equals_structured_kernels(dev, orc, name, f):
    h = qpath.qp_build_qubo(f, flags=qpath.QP_DENSE | qpath.QP_STRUCTURED)
    a = gpu_anneal(h, 16, 200, 3, kernel=qpath.QP_KERNEL_DENSE)
    for k in (qpath.QP_KERNEL_STRUCTURED, qpath.QP_KERNEL_STRUCTURED_ROWS, qpath.QP_KERNEL_STRUCTURED_FLAT,
              qpath.QP_KERNEL_STRUCTURED_GROUP):
        b = gpu_anneal(h, 16, 200, 3, kernel=k)
        for x, y in zip(a, b):
            assert (x == y).all()


@pytest.mark.parametrize("n", [5, 37, 300])
def test_dense_generic_qubo_with_frozen(dev, orc, n):
    rng = np.random.default_rng(n)
    Q = rng.integers(-60, 61, (n, n)).astype(np.int32)
    Q = np.triu(Q) + np.triu(Q, 1).T
    fr = (rng.random(n) < 0.1).astype(np.uint8)
    fv = (rng.random(n) < 0.5).astype(np.uint8)
    h = qpath.qp_build_from_dense(Q, c0=17, frozen=fr, frozen_val=fv)
    R, S = 24, 120
    ref = orc.anneal_dense(Q, 17, R, S, seed=99, T0=80.0, T1=0.5, frozen=fr, frozen_val=fv)
    assert_same(gpu_anneal(h, R, S, 99, T0=80.0, T1=0.5), ref)


def test_dense_int32_entries(dev, orc):
    rng = np.random.default_rng(3)
    n = 40
    Q = rng.integers(-100000, 100001, (n, n)).astype(np.int32)
    Q = np.triu(Q) + np.triu(Q, 1).T
    h = qpath.qp_build_from_dense(Q)
    ref = orc.anneal_dense(Q, 0, 8, 60, seed=4, T0=1e5, T1=10.0)
    assert_same(gpu_anneal(h, 8, 60, 4, T0=1e5, T1=10.0), ref)


def test_dense_h_in_global_memory(dev, orc):
    """n large enough that the local fields do not fit in shared memory."""
    f = inputs.obstacles(16, 16, 0.1, seed=3)
    P = problem(orc, f)
    assert P.n * 4 > 200 * 1024  # h plus the bitsets exceed the 227 KB limit
    S, c0 = P.dense()
    fr, fv = P.frozen()
    h = qpath.qp_build_qubo(f, flags=qpath.QP_DENSE)
    ref = orc.anneal_dense(S, c0, 2, 6, seed=8, frozen=fr, frozen_val=fv, C=P.C)
    assert_same(gpu_anneal(h, 2, 6, 8, kernel=qpath.QP_KERNEL_DENSE), ref)


# ----------------------------------------------------------------- decode
def test_decode_batch_and_single(dev, orc):
    import torch
    f = inputs.obstacles(5, 6, 0.1, seed=2)
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    st, E, B, A = gpu_anneal(h, 32, 1500, 4)
    rng = np.random.default_rng(1)
    others = [i for i in range(P.C) if i != P.start_cell]
    perm = [P.start_cell] + list(rng.permutation(others))
    xp = np.zeros((P.C, P.C), np.uint8)
    xp[np.arange(P.C), perm] = 1
    st = np.concatenate([st, xp.reshape(1, -1)])
    R = len(st)
    paths = torch.zeros((R, P.C), dtype=torch.int32, device="cuda")
    lens = torch.zeros(R, dtype=torch.int64, device="cuda")
    qpath.qp_decode_batch(h, R, torch.from_numpy(st).cuda(), paths, lens)
    torch.cuda.synchronize()
    paths, lens = paths.cpu().numpy(), lens.cpu().numpy()
    feasible = 0
    for r in range(R):
        ref = orc.decode(P.d, st[r])
        one = qpath.qp_decode_path(h, st[r])
        if ref is None:
            assert lens[r] == -1 and one is None
        else:
            feasible += 1
            assert lens[r] == ref[1] and (paths[r] == ref[0]).all()
            assert one[1] == ref[1] and (one[0] == ref[0]).all()
    assert feasible >= 1 and lens[-1] >= 0


# ----------------------------------------------------------------- errors
def test_errors_are_statuses(dev):
    import torch
    bad = inputs.Field(3, 3, np.array([0, 1, 1, 1, 1, 1, 1, 1, 1], np.uint8), 0)
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_build_qubo(bad)
    assert e.value.status == qpath.QP_EINVAL
    with pytest.raises(qpath.QpError):
        qpath.qp_build_qubo(inputs.rect(1, 1))
    h = qpath.qp_build_qubo(inputs.rect(3, 3))
    st = torch.zeros((2, 81), dtype=torch.uint8, device="cuda")
    E = torch.zeros(2, dtype=torch.int64, device="cuda")
    for sc in [qpath.schedule(10, 1e3, 1.0, 5, 3), qpath.schedule(0), qpath.schedule(10, -1.0, 1.0)]:
        with pytest.raises(qpath.QpError) as e:
            qpath.qp_anneal(h, 2, sc, 1, None, st, E)
        assert e.value.status == qpath.QP_EINVAL
    with pytest.raises(qpath.QpError):
        qpath.qp_anneal(h, 0, qpath.schedule(10), 1, None, st, E)
    with pytest.raises(qpath.QpError):
        qpath.qp_anneal_ex(h, 2, qpath.schedule(10), 1, None, st, E, kernel=qpath.QP_KERNEL_DENSE)
    big = inputs.rect(7, 7)
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_build_qubo(big, A=10 ** 9)
    assert e.value.status == qpath.QP_ERANGE


# ----------------------------------------------------------------- full-size workloads, sampled
@pytest.mark.slow
def test_full_size_10x10_structured_sampled(dev, orc):
    """10x10 field, 10% obstacles (seed 1), 1024 replicas x 5000 sweeps,
    geometric 1e3 -> 1, seed 1 -- the benchmark's launch -- with the oracle on
    sampled replicas."""
    w = inputs.WORKLOADS["10x10-p0.10"]
    f = w["field"]()
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    got = gpu_anneal(h, w["replicas"], w["n_sweeps"], w["seed"])
    idx = [0, 1, 511, 1023]
    ref = orc.anneal_structured(P, idx, w["n_sweeps"], seed=w["seed"])
    assert_same(got, ref, idx)
    feas = got[2] < qpath.E_NONE
    assert feas.mean() > 0.5


@pytest.mark.slow
def test_full_size_10x10_dense_sampled(dev, orc):
    w = inputs.WORKLOADS["10x10-p0.10"]
    f = w["field"]()
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f, flags=qpath.QP_DENSE | qpath.QP_STRUCTURED)
    got = gpu_anneal(h, w["replicas"], w["n_sweeps"], w["seed"], kernel=qpath.QP_KERNEL_DENSE)
    idx = [3, 700]
    ref = orc.anneal_structured(P, idx, w["n_sweeps"], seed=w["seed"])
    assert_same(got, ref, idx)


@pytest.mark.parametrize("name,f,R,S", [("6x6-p0.2", inputs.obstacles(6, 6, 0.2, seed=3, start=14), 40, 3000),
                                         ("3x5-start7", inputs.rect(3, 5, start=7), 33, 1500),
                                         ("13x13-p0.1", inputs.obstacles(13, 13, 0.1, seed=5, start=20), 6, 1200)])
def test_skip_settled_same_results(dev, orc, name, f, R, S):
    """Whole schedules (cooling to T = 1, so replicas settle): skipping settled
    sweeps changes nothing, against the oracle and against the full kernel."""
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    import torch
    n = P.n
    outs = []
    for flags in (0, qpath.QP_ANNEAL_SKIP_SETTLED):
        st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
        E = torch.zeros(R, dtype=torch.int64, device="cuda")
        B = torch.zeros(R, dtype=torch.int64, device="cuda")
        A = torch.zeros(R, dtype=torch.int64, device="cuda")
        qpath.qp_anneal_ex(h, R, qpath.schedule(S), 9, None, st, E, B, kernel=qpath.QP_KERNEL_STRUCTURED_ROWS,
                           accepts_out=A, flags=flags, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        outs.append((st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy(), A.cpu().numpy()))
    for a, b in zip(outs[0], outs[1]):
        assert (a == b).all()
    idx = [0, R - 1]
    ref = orc.anneal_structured(P, idx, S, seed=9)
    assert_same(outs[1], ref, idx)


@pytest.mark.parametrize("rpc", [4, 5])
def test_dense_row_staging_modes(dev, orc, rpc):
    """The 10x10 field's dense sweep (n = 8464) with 4 replicas per CTA stages
    accepted rows by bulk copy into shared memory; with 5 the row buffers no
    longer fit and rows stream through registers.  Both match the oracle."""
    f = inputs.WORKLOADS["10x10-p0.10"]["field"]()
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f, flags=qpath.QP_DENSE | qpath.QP_STRUCTURED)
    R = 11
    got = gpu_anneal(h, R, 40, 5, T0=2000.0, T1=500.0, kernel=qpath.QP_KERNEL_DENSE, rpc=rpc)
    ref = orc.anneal_structured(P, R, 40, T0=2000.0, T1=500.0, seed=5)
    assert_same(got, ref)
    assert ref.accepts.min() > 1000  # many rows staged per replica


@pytest.mark.slow
def test_full_size_24x24_structured_sampled(dev, orc):
    """24x24 field, 15% obstacles, 4096 replicas x 10000 sweeps, int16 d; two
    sampled replicas through the oracle (about a minute of CPU each)."""
    w = inputs.WORKLOADS["24x24-p0.15"]
    f = w["field"]()
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f, flags=qpath.QP_STRUCTURED | qpath.QP_DIST_I16)
    got = gpu_anneal(h, w["replicas"], w["n_sweeps"], w["seed"])
    idx = [0, 4095]
    ref = orc.anneal_structured(P, idx, w["n_sweeps"], seed=w["seed"])
    assert_same(got, ref, idx)


@pytest.mark.parametrize("shape,p,seed,R", [((8, 8), 0.0, 1, 7), ((7, 9), 0.1, 2, 13), ((11, 11), 0.05, 3, 9),
                                           ((2, 3), 0.0, 4, 5)])
def test_grouped_kernel_partial_warps(dev, orc, shape, p, seed, R):
    """Group sizes 4 (C <= 64) and 2 (C <= 128) with replica counts that leave
    idle groups in the last warp."""
    f = inputs.obstacles(*shape, p, seed=seed)
    P = problem(orc, f)
    h = qpath.qp_build_qubo(f)
    ref = orc.anneal_structured(P, R, 120, seed=seed)
    assert_same(gpu_anneal(h, R, 120, seed, kernel=qpath.QP_KERNEL_STRUCTURED_GROUP), ref)
