"""Caller-owned device buffers that are too small are refused before any
launch (QP_EINVAL): the library asks the driver for the allocation holding
each pointer (cuMemGetAddressRange) and checks that the bytes the call writes
fit in it.  Nothing is launched on a refused call, so nothing faults, and a
correct call afterwards still matches the oracle.  (A pooling allocator hands
out buffers inside larger blocks; only overruns past the block are visible,
so the buffers here are large and freshly allocated.)"""
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


def test_undersized_device_outputs_are_refused(dev):
    import torch
    import oracle
    f = inputs.WORKLOADS["10x10-p0.10"]["field"]()
    h = qpath.qp_build_qubo(f)
    n, C = h.info["n"], h.info["C"]
    R = 4096
    sc = qpath.schedule(20)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    short = torch.zeros((R - 2048, n), dtype=torch.uint8, device="cuda")  # 17 MB short
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_anneal_ex(h, R, sc, 1, None, short, E, stream=torch.cuda.current_stream())
    assert e.value.status == qpath.QP_EINVAL and "states_out" in str(e.value)
    # the same buffer as the input of a decode of R states
    paths = torch.zeros((R, C), dtype=torch.int32, device="cuda")
    lens = torch.zeros(R, dtype=torch.int64, device="cuda")
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_decode_batch(h, R, short, paths, lens, stream=torch.cuda.current_stream())
    assert e.value.status == qpath.QP_EINVAL
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_repair_batch(h, R, short, 0, paths, lens, stream=torch.cuda.current_stream())
    assert e.value.status == qpath.QP_EINVAL
    # nothing ran; a call that fits works and matches the oracle
    R2 = R - 2048
    qpath.qp_anneal_ex(h, R2, sc, 1, None, short, E, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start)
    idx = [0, 777, R2 - 1]
    ref = oracle.anneal_structured(P, idx, 20, seed=1)
    assert (E.cpu().numpy()[idx] == ref.energies).all()
    assert (short.cpu().numpy()[idx] == ref.states).all()
