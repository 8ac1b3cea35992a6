"""The schedule-table cache drops its least recently used schedules beyond its
size limit (here shrunk through QPATH_SCHEDULE_CACHE_MB), while a batch keeps
the tables its captured graph points to: replaying it after its schedule left
the cache still gives the per-field results; an allocation-free call, which
needs the tables cached, reports their absence."""
import os

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


def test_evicted_schedule_survives_in_a_batch(dev, monkeypatch):
    import torch
    monkeypatch.setenv("QPATH_SCHEDULE_CACHE_MB", "1")
    fields = inputs.batch(4, seed=77)
    hs = [qpath.qp_build_qubo(f) for f in fields]
    R, seed = 6, 5
    sc = qpath.schedule(1500, 777.0, 1.5)  # ~18 MB of tables: above the 1 MB limit on its own
    st = [torch.zeros((R, h.info["n"]), dtype=torch.uint8, device="cuda") for h in hs]
    E = [torch.zeros(R, dtype=torch.int64, device="cuda") for _ in hs]
    B = [torch.zeros(R, dtype=torch.int64, device="cuda") for _ in hs]
    b = qpath.qp_batch_create(hs, R, sc, seed, st, E, B)
    # other schedules push it out of the cache
    h0 = hs[0]
    n0 = h0.info["n"]
    tmp = torch.zeros((R, n0), dtype=torch.uint8, device="cuda")
    tE = torch.zeros(R, dtype=torch.int64, device="cuda")
    for k in range(3):
        qpath.qp_anneal(h0, R, qpath.schedule(1200 + k, 900.0, 2.0), 1, None, tmp, tE,
                        stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    with pytest.raises(qpath.QpError):  # the tables are no longer cached
        qpath.qp_anneal_noalloc(h0, R, sc, seed, None, tmp, tE)
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    for f, h in enumerate(hs):
        s2 = torch.zeros((R, h.info["n"]), dtype=torch.uint8, device="cuda")
        e2 = torch.zeros(R, dtype=torch.int64, device="cuda")
        b2 = torch.zeros(R, dtype=torch.int64, device="cuda")
        qpath.qp_anneal(h, R, sc, seed + f, None, s2, e2, b2, stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert torch.equal(st[f], s2) and torch.equal(E[f], e2) and torch.equal(B[f], b2), f
    b.close()
