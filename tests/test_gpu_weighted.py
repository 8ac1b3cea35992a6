"""The extended objective on the GPU (per-leg weights on the distance term):
the dense form the device builds against the oracle's, the dense anneal of a
weighted handle against the oracle's anneal of that form bit for bit, equal
weights against the unweighted handle, the structured calls refused, and the
weighted optimum of a small field found."""
import itertools

import numpy as np
import pytest

from conftest import has_gpu
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, objectives, qpath

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    qpath.lib()


def gpu_anneal(h, R, S, seed, T0=1e3, T1=1.0):
    import torch
    n = h.info["n"]
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    A = torch.zeros(R, dtype=torch.int64, device="cuda")
    qpath.qp_anneal_ex(h, R, qpath.schedule(S, T0, T1), seed, None, st, E, B, accepts_out=A,
                       stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy(), A.cpu().numpy()


def clamp_bits(C, s):
    fr = np.zeros((C, C), np.uint8)
    fv = np.zeros((C, C), np.uint8)
    fr[0, :] = 1
    fr[:, s] = 1
    fv[0, s] = 1
    return fr.reshape(-1), fv.reshape(-1)


FIELDS = [("3x3", inputs.rect(3, 3)), ("4x5-p0.2", inputs.obstacles(4, 5, 0.2, seed=2, start=6)),
          ("6x6-p0.1", inputs.obstacles(6, 6, 0.1, seed=4, start=9))]


@pytest.mark.parametrize("name,f", FIELDS)
def test_weighted_dense_form_and_anneal_match_the_oracle(dev, orc, name, f):
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    C = P.C
    w = objectives.payload_leg_weights(C, 20, 3)
    h = qpath.qp_build_qubo_weighted(f, w)
    info = qpath.qp_qubo_info(h)
    assert info["A"] == 2 * int(w.max()) * int(P.d.max())
    S_ref, c0_ref = orc.dense_qubo_weighted(P.d, info["A"], w)
    assert info["c0"] == c0_ref
    assert np.array_equal(qpath.qp_export_dense(h), S_ref)
    R, S = 16, 400
    got = gpu_anneal(h, R, S, seed=7, T0=3e4, T1=5.0)
    fr, fv = clamp_bits(C, P.start_cell)
    ref = orc.anneal_dense(S_ref, c0_ref, R, S, seed=7, T0=3e4, T1=5.0, frozen=fr, frozen_val=fv, C=C)
    st, E, B, A = got
    assert (E == ref.energies).all() and (B == ref.best).all() and (A == ref.accepts).all()
    assert (st == ref.states).all()


def test_equal_weights_equal_the_unweighted_handle(dev, orc):
    f = inputs.obstacles(5, 5, 0.15, seed=1)
    C = qpath.qp_build_qubo(f).info["C"]
    hw = qpath.qp_build_qubo_weighted(f, np.full(C - 1, 2, np.int32), A=900)
    hu = qpath.qp_build_qubo(f, A=900, B=2, flags=qpath.QP_DENSE | qpath.QP_STRUCTURED)
    assert np.array_equal(qpath.qp_export_dense(hw), qpath.qp_export_dense(hu))
    a = gpu_anneal(hw, 8, 300, 3)
    b = gpu_anneal(hu, 8, 300, 3)  # the structured kernel on the unweighted handle
    for x, y in zip(a, b):
        assert (x == y).all()


def test_structured_calls_refuse_a_weighted_handle(dev):
    import torch
    f = inputs.rect(3, 4)
    h = qpath.qp_build_qubo_weighted(f, objectives.payload_leg_weights(12, 5, 1))
    n = h.info["n"]
    st = torch.zeros((4, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(qpath.QpError):
        qpath.qp_anneal_ex(h, 4, qpath.schedule(10), 1, None, st, E, kernel=qpath.QP_KERNEL_STRUCTURED)
    paths = torch.zeros((4, 12), dtype=torch.int32, device="cuda")
    lens = torch.zeros(4, dtype=torch.int64, device="cuda")
    with pytest.raises(qpath.QpError):
        qpath.qp_repair_batch(h, 4, st, -1, paths, lens)
    with pytest.raises(qpath.QpError):
        qpath.qp_build_qubo_weighted(f, np.ones(5, np.int32))  # C - 1 = 11 weights needed
    with pytest.raises(qpath.QpError):
        qpath.qp_build_qubo_weighted(f, -np.ones(11, np.int32))


def test_weighted_optimum_of_a_small_field(dev, orc):
    """2 x 3 field: the best energy over the replicas is the cheapest weighted
    path by brute force over all 120 paths, and it decodes to such a path."""
    f = inputs.rect(2, 3)
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    C, s, d = P.C, P.start_cell, P.d
    w = objectives.payload_leg_weights(C, 2, 5)  # heavy first legs
    costs = {p: objectives.flight_energy((s,) + p, d, w)
             for p in itertools.permutations([c for c in range(C) if c != s])}
    opt = min(costs.values())
    h = qpath.qp_build_qubo_weighted(f, w)
    st, E, B, A = gpu_anneal(h, 256, 2000, 11, T0=2e4, T1=1.0)
    assert B.min() == opt
    r = int(np.argmin(E))
    assert E[r] == opt
    path, _ = qpath.qp_decode_path(h, st[r])
    assert objectives.flight_energy(path, d, w) == opt
