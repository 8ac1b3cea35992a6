"""The allocation-free structured anneal, qp_anneal_noalloc, for callers that
cannot allocate device memory while they run (software that reserves all of
its memory at start-up, or runs under a memory manager that owns the GPU).

It must return exactly what qp_anneal_ex returns with the same kernel, on two
calls in a row (the second call reuses the library's fixed scratch array that
the first one filled).  This file is collected last so that a run stopping at
the first failure has run every other test first; it also passes alone in a
fresh process, because it builds the schedule tables it needs itself.
"""
import numpy as np
import pytest

from conftest import has_gpu
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath

pytestmark = pytest.mark.gpu


def _run(fn, h, R, sc, seed, offset, init=None):
    import torch
    n = h.info["n"]
    st = torch.full((R, n), 7, dtype=torch.uint8, device="cuda")
    E = torch.full((R,), -5, dtype=torch.int64, device="cuda")
    B = torch.full((R,), -5, dtype=torch.int64, device="cuda")
    if fn == "ex":
        qpath.qp_anneal_ex(h, R, sc, seed, init, st, E, B, kernel=qpath.QP_KERNEL_STRUCTURED_FLAT,
                           replica_offset=offset, stream=torch.cuda.current_stream())
    else:
        qpath.qp_anneal_noalloc(h, R, sc, seed, init, st, E, B, replica_offset=offset,
                                stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy()


def test_noalloc_matches_anneal_ex_on_two_calls():
    if not has_gpu():
        pytest.skip("no CUDA device")
    import torch
    qbuild.build()
    # 18x18 with 10% obstacles: more than 256 cells, so the kernel keeps each
    # replica's spins in the scratch array rather than in shared memory
    f = inputs.obstacles(18, 18, 0.1, seed=8, start=5)
    h = qpath.qp_build_qubo(f)
    assert h.info["C"] > 256
    sc = qpath.schedule(60, 1e3, 1.0)
    calls = [(6, 11, 0, None), (9, 12, 40, None)]
    rng = np.random.default_rng(3)
    init = (rng.random((5, h.info["n"])) < 0.01).astype(np.uint8)
    calls.append((5, 13, 7, torch.from_numpy(init).cuda()))
    for R, seed, offset, ini in calls:
        ref = _run("ex", h, R, sc, seed, offset, ini)  # also builds the schedule's tables
        got = _run("noalloc", h, R, sc, seed, offset, ini)
        for a, b in zip(got, ref):
            assert (a == b).all()
    # beyond the fixed scratch size the call is refused, not truncated
    n = h.info["n"]
    big = 1 + (16 << 20) // (4 * ((n + 31) // 32 + 1))  # per-replica words >= ceil(n/32) + 1
    st = torch.zeros((big, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(big, dtype=torch.int64, device="cuda")
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_anneal_noalloc(h, big, sc, 1, None, st, E)
    assert e.value.status == qpath.QP_ERANGE
    # host buffers are refused
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_anneal_noalloc(h, 2, sc, 1, None, np.zeros((2, n), np.uint8), np.zeros(2, np.int64))
    assert e.value.status == qpath.QP_EINVAL
