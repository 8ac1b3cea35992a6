"""GPU parity of replica exchange (qp_anneal_pt) against the CPU reference
(oracle/pt_ref.py): final states, energies, best feasible energies, levels
and trade counts, bit for bit, for the same seed."""
import numpy as np
import pytest

from conftest import has_gpu
from oracle import pt_ref
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


def gpu_pt(h, G, M, T_lo, T_hi, I, rounds, seed, init=None, host=False):
    import torch
    n = h.info["n"]
    R = G * M
    pt = qpath.pt_schedule(M, T_lo, T_hi, I, rounds)
    if host:
        out = dict(states=np.zeros((R, n), np.uint8), energies=np.zeros(R, np.int64),
                   best=np.zeros(R, np.int64), levels=np.zeros(R, np.int32),
                   swaps=np.zeros(G * (M - 1), np.int64))
        qpath.qp_anneal_pt(h, G, pt, seed, init, out["states"], out["energies"], out["best"], out["levels"],
                           out["swaps"])
        return out
    t = dict(states=torch.zeros((R, n), dtype=torch.uint8, device="cuda"),
             energies=torch.zeros(R, dtype=torch.int64, device="cuda"),
             best=torch.zeros(R, dtype=torch.int64, device="cuda"),
             levels=torch.zeros(R, dtype=torch.int32, device="cuda"),
             swaps=torch.zeros(G * (M - 1), dtype=torch.int64, device="cuda"))
    ini = None if init is None else torch.from_numpy(np.ascontiguousarray(init)).cuda()
    qpath.qp_anneal_pt(h, G, pt, seed, ini, t["states"], t["energies"], t["best"], t["levels"], t["swaps"],
                       stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in t.items()}


def assert_same(got, ref):
    assert (got["energies"] == ref["energies"]).all(), (got["energies"][:8], ref["energies"][:8])
    assert (got["best"] == ref["best"]).all()
    assert (got["levels"] == ref["levels"]).all()
    assert (got["swaps"] == ref["swaps"]).all()
    assert (got["states"] == ref["states"]).all()


CASES = [
    # name, field, G, M, T_lo, T_hi, I, rounds
    ("4x4", inputs.rect(4, 4), 6, 4, 10.0, 1000.0, 5, 6),
    ("6x6-p0.2-odd-M", inputs.obstacles(6, 6, 0.2, seed=3, start=14), 3, 5, 20.0, 800.0, 3, 7),
    ("10x10-p0.1", inputs.obstacles(10, 10, 0.1, seed=1), 2, 8, 5.0, 1000.0, 2, 4),
]


@pytest.mark.parametrize("name,f,G,M,T_lo,T_hi,I,rounds", CASES)
def test_pt_parity(dev, orc, name, f, G, M, T_lo, T_hi, I, rounds):
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    h = qpath.qp_build_qubo(f)
    ref = pt_ref.anneal_pt(P, G, M, T_lo, T_hi, I, rounds, seed=11)
    assert ref["swaps"].sum() > 0
    assert_same(gpu_pt(h, G, M, T_lo, T_hi, I, rounds, 11), ref)
    assert_same(gpu_pt(h, G, M, T_lo, T_hi, I, rounds, 11, host=True), ref)


def test_pt_parity_with_init_states(dev, orc):
    f = inputs.rect(3, 5, start=7)
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    G, M = 4, 3
    rng = np.random.Generator(np.random.PCG64(4))
    init = (rng.random((G * M, P.n)) < 0.1).astype(np.uint8)
    h = qpath.qp_build_qubo(f)
    ref = pt_ref.anneal_pt(P, G, M, 30.0, 600.0, 4, 5, seed=2, init_states=init)
    assert_same(gpu_pt(h, G, M, 30.0, 600.0, 4, 5, 2, init=init), ref)


def test_pt_parity_flat_kernel_above_512_cells(dev, orc):
    f = inputs.obstacles(24, 24, 0.05, seed=8)
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    assert P.C > 512
    h = qpath.qp_build_qubo(f)
    ref = pt_ref.anneal_pt(P, 1, 2, 100.0, 1000.0, 1, 2, seed=5)
    assert_same(gpu_pt(h, 1, 2, 100.0, 1000.0, 1, 2, 5), ref)


def test_pt_rejects_bad_ladders(dev):
    h = qpath.qp_build_qubo(inputs.rect(3, 3))
    import torch
    st = torch.zeros((4, 81), dtype=torch.uint8, device="cuda")
    E = torch.zeros(4, dtype=torch.int64, device="cuda")
    for pt in [qpath.pt_schedule(1, 1.0, 2.0, 1, 1), qpath.pt_schedule(2, 5.0, 5.0, 1, 1),
               qpath.pt_schedule(2, 1.0, 2.0, 0, 1), qpath.pt_schedule(2, 1.0, 2.0, 1, 0)]:
        with pytest.raises(qpath.QpError):
            qpath.qp_anneal_pt(h, 2, pt, 1, None, st, E)
