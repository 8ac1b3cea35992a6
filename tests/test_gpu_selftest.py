"""The bounded wait that guards the library's asynchronous copies gives up
instead of hanging: a wait on an mbarrier phase that nothing completes comes
back with "timed out" after its bound, and the context keeps working."""
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


def test_wait_on_a_phase_that_never_completes_times_out(dev, orc):
    r = qpath.qp_selftest_wait()
    assert r["timed_out"] == 1
    assert 100.0 < r["waited_ms"] < 5000.0, r
    # the context is still usable: a small anneal matches the oracle
    import torch
    f = inputs.rect(3, 4)
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    h = qpath.qp_build_qubo(f)
    R, S = 8, 50
    st = torch.zeros((R, P.n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    qpath.qp_anneal(h, R, qpath.schedule(S), 4, None, st, E, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    ref = orc.anneal_structured(P, R, S, seed=4)
    assert (E.cpu().numpy() == ref.energies).all()
