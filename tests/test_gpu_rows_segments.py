"""The row kernel with the spins in global memory, run persistent over
(replica, sweep segment) units when there are more chains than fit on the GPU
at once: every replica's states, energies, best energies and accept counts
equal the shared-memory-spins kernel's (one launch, whole chains), and sampled
replicas equal the oracle."""
import numpy as np
import pytest

from conftest import has_gpu
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    qpath.lib()


def _run(h, R, sc, seed, kernel):
    import torch
    n = h.info["n"]
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    acc = torch.zeros(R, dtype=torch.int64, device="cuda")
    qpath.qp_anneal_ex(h, R, sc, seed, None, st, E, B, kernel=kernel, accepts_out=acc,
                       stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st, E, B, acc


@pytest.mark.parametrize("n_sweeps,begin", [(1200, 0), (2600, 1300)])
def test_segmented_chains_equal_whole_chains(dev, n_sweeps, begin):
    import oracle
    import torch
    f = inputs.obstacles(18, 18, 0.1, seed=8, start=5)  # 292 cells
    h = qpath.qp_build_qubo(f)
    C = h.info["C"]
    assert 256 < C <= 512
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    R = 16 * sms + 37  # more chains than fit at once (at most 12 per SM)
    sc = qpath.schedule(n_sweeps, sweep_begin=begin, sweep_end=n_sweeps)
    got = _run(h, R, sc, 7, qpath.QP_KERNEL_STRUCTURED)
    ref = _run(h, R, sc, 7, qpath.QP_KERNEL_STRUCTURED_ROWS_SHARED)
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start)
    idx = [0, R // 2, R - 1]
    o = oracle.anneal_structured(P, idx, n_sweeps, seed=7, sweep_begin=begin, sweep_end=n_sweeps)
    assert (got[1].cpu().numpy()[idx] == o.energies).all()
    assert (got[2].cpu().numpy()[idx] == o.best).all()
    assert (got[0].cpu().numpy()[idx] == o.states).all()
