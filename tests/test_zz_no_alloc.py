"""The allocation-free structured anneal, qp_anneal_noalloc, for callers that
cannot allocate device memory while they run (software that reserves all of
its memory at start-up, or runs under a memory manager that owns the GPU).

It must return exactly what qp_anneal_ex returns with the same kernel, on two
calls in a row (the second call reuses the library's fixed scratch array that
the first one filled), and a call must allocate nothing: with every library
allocation made to fail (QPATH_FAIL_ALLOC=0) it still succeeds, and the
device's free memory is the same before and after it.  This file is collected
last so that a run stopping at the first failure has run every other test
first; it also passes alone in a fresh process, because it builds the
schedule tables it needs itself.
"""
import os

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
    # one more call with every library allocation refused and the device's
    # free memory watched: it allocates nothing, and still matches
    R, seed, offset = 7, 21, 3
    ref = _run("ex", h, R, sc, seed, offset)
    n = h.info["n"]
    st = torch.full((R, n), 7, dtype=torch.uint8, device="cuda")
    E = torch.full((R,), -5, dtype=torch.int64, device="cuda")
    B = torch.full((R,), -5, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    old = os.environ.get("QPATH_FAIL_ALLOC")
    os.environ["QPATH_FAIL_ALLOC"] = "0"
    try:
        qpath.qp_anneal_noalloc(h, R, sc, seed, None, st, E, B, replica_offset=offset,
                                stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        # the hook is live: an entry point that does allocate fails now
        with pytest.raises(qpath.QpError) as e:
            qpath.qp_build_qubo(inputs.obstacles(6, 6, 0.1, seed=1))
        assert e.value.status == qpath.QP_ENOMEM
    finally:
        if old is None:
            del os.environ["QPATH_FAIL_ALLOC"]
        else:
            os.environ["QPATH_FAIL_ALLOC"] = old
    assert free1 == free0
    for a, b in zip((st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy()), ref):
        assert (a == b).all()
    # beyond the fixed scratch size the call is refused, not truncated
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
