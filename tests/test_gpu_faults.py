"""Failure injection on the host: device allocations made to fail one after
another (the library's QPATH_FAIL_ALLOC hook), so that every allocation site
of a pipeline covering all entry points is hit once.  Each call must return
QP_ENOMEM as a status (no crash, no launch on a missing buffer), and the
library must work normally afterwards: the same pipeline then matches the
CPU oracle bit for bit.  Nothing on the GPU is made to fault."""
import os

import numpy as np
import pytest

from conftest import has_gpu
import oracle
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath

pytestmark = pytest.mark.gpu

R, S = 32, 40


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    oracle.build()
    qpath.lib()


def pipeline(k):
    """Every allocating entry point once; a fresh schedule and ladder per call
    (key k) so that the process-wide table caches allocate too."""
    import torch
    f = inputs.obstacles(6, 6, 0.15, seed=2)
    h = qpath.qp_build_qubo(f, flags=qpath.QP_STRUCTURED | qpath.QP_DENSE)
    n, C = h.info["n"], h.info["C"]
    sc = qpath.schedule(S, 1000.0 + k, 1.0)
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream()
    qpath.qp_anneal(h, R, sc, 3, None, st, E, B, stream=s)
    stn, En = np.zeros((R, n), np.uint8), np.zeros(R, np.int64)
    qpath.qp_anneal_ex(h, R, sc, 3, None, stn, En, kernel=qpath.QP_KERNEL_DENSE)
    paths = torch.zeros((R, C), dtype=torch.int32, device="cuda")
    lens = torch.zeros(R, dtype=torch.int64, device="cuda")
    qpath.qp_repair_batch(h, R, st, -1, paths, lens, stream=s)
    pst, pE = np.zeros((8, n), np.uint8), np.zeros(8, np.int64)
    qpath.qp_anneal_pt(h, 2, qpath.pt_schedule(4, 10.0 + k % 500, 1000.0, 5, 2), 3, None, pst, pE)
    h2 = qpath.qp_build_qubo(inputs.obstacles(5, 7, 0.1, seed=3))
    outs = [torch.zeros((16, hh.info["n"]), dtype=torch.uint8, device="cuda") for hh in (h, h2)]
    eouts = [torch.zeros(16, dtype=torch.int64, device="cuda") for _ in (h, h2)]
    qpath.qp_anneal_batch([h, h2], 16, sc, 5, outs, eouts, stream=s)
    m = qpath.WarmStartModel(seed=1)
    X = qpath.qp_ws_features(f)
    qpath.qp_ws_forward(m, X)
    qpath.qp_ws_train_step(m, X, np.arange(C, dtype=np.int32), np.full(C, C, np.int32), 1e-3)
    torch.cuda.synchronize()
    return f, st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy(), stn, En


def test_allocation_failures_are_statuses(dev, monkeypatch):
    failed, k = 0, 0
    for k in range(400):
        monkeypatch.setenv("QPATH_FAIL_ALLOC", str(k))
        try:
            pipeline(k)
        except qpath.QpError as e:
            assert e.status == qpath.QP_ENOMEM, (k, str(e))
            failed += 1
            continue
        break  # k allocations cover the whole pipeline
    else:
        pytest.fail("the pipeline never completed")
    assert failed == k and failed > 20, (failed, k)  # every allocation site was hit once
    print(f"{failed} allocation sites failed one by one")
    monkeypatch.delenv("QPATH_FAIL_ALLOC")
    f, st, E, B, stn, En = pipeline(10_000)
    P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start)
    ref = oracle.anneal_structured(P, R, S, seed=3, T0=1000.0 + 10_000)
    assert (E == ref.energies).all() and (B == ref.best).all() and (st == ref.states).all()
    assert (En == ref.energies).all() and (stn == ref.states).all()
