"""Calls on different handles from several host threads at once (the binding
releases the interpreter lock during each call): fields of different sizes,
so the launches need different shared-memory limits, each on its own stream;
every result still equals the CPU oracle's."""
import threading

import numpy as np
import pytest

from conftest import has_gpu
import oracle
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    oracle.build()
    qpath.lib()


def test_concurrent_calls_on_separate_handles(dev):
    import torch
    cases = [(inputs.obstacles(6, 6, 0.2, seed=3, start=14), 32, 60, qpath.QP_KERNEL_STRUCTURED_ROWS),
             (inputs.obstacles(13, 13, 0.1, seed=5, start=20), 24, 20, qpath.QP_KERNEL_STRUCTURED_ROWS),
             (inputs.obstacles(18, 18, 0.1, seed=8, start=5), 4, 4, qpath.QP_KERNEL_STRUCTURED_ROWS),
             (inputs.obstacles(5, 5, 0.1, seed=4), 32, 60, qpath.QP_KERNEL_DENSE)]
    out = [None] * len(cases)
    errors = []

    def work(i):
        try:
            f, R, S, kernel = cases[i]
            flags = qpath.QP_STRUCTURED | (qpath.QP_DENSE if kernel == qpath.QP_KERNEL_DENSE else 0)
            h = qpath.qp_build_qubo(f, flags=flags)
            n = h.info["n"]
            s = torch.cuda.Stream()
            res = []
            for rep in range(3):
                st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
                E = torch.zeros(R, dtype=torch.int64, device="cuda")
                with torch.cuda.stream(s):
                    qpath.qp_anneal_ex(h, R, qpath.schedule(S), 7, None, st, E, kernel=kernel, stream=s)
                s.synchronize()
                res.append((st.cpu().numpy(), E.cpu().numpy()))
            out[i] = res
            h.close()
        except Exception as e:  # reported below, on the main thread
            errors.append((i, repr(e)))

    threads = [threading.Thread(target=work, args=(i,)) for i in range(len(cases))]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for i, (f, R, S, kernel) in enumerate(cases):
        P = oracle.Problem(f.rows, f.cols, f.free_mask, f.start)
        ref = oracle.anneal_structured(P, R, S, seed=7)
        for st, E in out[i]:
            assert (E == ref.energies).all() and (st == ref.states).all(), i
