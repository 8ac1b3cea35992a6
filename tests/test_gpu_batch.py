"""Batched persistent anneal (many uneven fields, one CUDA-graph launch) vs the
per-field anneal and the CPU oracle, bit for bit."""
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


def outputs(handles, R):
    import torch
    st = [torch.full((R, h.info["n"]), 9, dtype=torch.uint8, device="cuda") for h in handles]
    E = [torch.full((R,), -3, dtype=torch.int64, device="cuda") for _ in handles]
    B = [torch.full((R,), -3, dtype=torch.int64, device="cuda") for _ in handles]
    return st, E, B


def single(h, R, sc, seed):
    import torch
    n = h.info["n"]
    st = torch.zeros((R, n), dtype=torch.uint8, device="cuda")
    E = torch.zeros(R, dtype=torch.int64, device="cuda")
    B = torch.zeros(R, dtype=torch.int64, device="cuda")
    qpath.qp_anneal(h, R, sc, seed, None, st, E, B, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return st.cpu().numpy(), E.cpu().numpy(), B.cpu().numpy()


def check_fields(handles, R, sc, seed, st, E, B, fields=None):
    for f in (range(len(handles)) if fields is None else fields):
        ref = single(handles[f], R, sc, seed + f)
        assert (st[f].cpu().numpy() == ref[0]).all(), f
        assert (E[f].cpu().numpy() == ref[1]).all(), f
        assert (B[f].cpu().numpy() == ref[2]).all(), f


def test_batch_equals_per_field_and_oracle(dev, orc):
    import torch
    fields = inputs.batch(12, seed=5)
    handles = [qpath.qp_build_qubo(f) for f in fields]
    R, seed = 16, 77
    sc = qpath.schedule(150)
    st, E, B = outputs(handles, R)
    b = qpath.qp_batch_create(handles, R, sc, seed, st, E, B)
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_fields(handles, R, sc, seed, st, E, B)
    for f in (0, 7):
        fl = fields[f]
        P = orc.Problem(fl.rows, fl.cols, fl.free_mask, fl.start)
        ref = orc.anneal_structured(P, R, 150, seed=seed + f)
        assert (st[f].cpu().numpy() == ref.states).all()
        assert (E[f].cpu().numpy() == ref.energies).all()
        assert (B[f].cpu().numpy() == ref.best).all()
    # replaying the graph reproduces the results exactly
    for x in st:
        x.fill_(5)
    for x in E:
        x.fill_(0)
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_fields(handles, R, sc, seed, st, E, B, fields=[0, 11])
    b.close()


@pytest.mark.parametrize("rpc,ctas", [(1, 1), (2, 3), (8, 0), (16, 0)])
def test_batch_configurations(dev, rpc, ctas):
    """A few CTAs force every warp to take many units from the queue."""
    import torch
    fields = inputs.batch(6, seed=9)
    handles = [qpath.qp_build_qubo(f) for f in fields]
    R, seed = 5, 3
    sc = qpath.schedule(60)
    st, E, B = outputs(handles, R)
    b = qpath.qp_batch_create(handles, R, sc, seed, st, E, B, replicas_per_cta=rpc, ctas=ctas)
    info = b.info
    assert info["units"] == 6 * R
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_fields(handles, R, sc, seed, st, E, B)


def test_batch_skip_settled_same_results(dev):
    """A whole cooling schedule, settled sweeps skipped: same as the full run."""
    import torch
    fields = inputs.batch(10, seed=31)
    handles = [qpath.qp_build_qubo(f) for f in fields]
    R, seed = 12, 8
    sc = qpath.schedule(1500)
    st, E, B = outputs(handles, R)
    b = qpath.qp_batch_create(handles, R, sc, seed, st, E, B, flags=qpath.QP_ANNEAL_SKIP_SETTLED)
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_fields(handles, R, sc, seed, st, E, B)
    b.close()


def test_batch_mixed_sizes_up_to_512_cells(dev):
    import torch
    fields = [inputs.rect(3, 3), inputs.obstacles(18, 18, 0.1, seed=8, start=5), inputs.rect(1, 2),
              inputs.obstacles(12, 13, 0.1, seed=1)]
    handles = [qpath.qp_build_qubo(f) for f in fields]
    assert max(h.info["C"] for h in handles) > 256
    R, seed = 3, 21
    sc = qpath.schedule(10)
    st, E, B = outputs(handles, R)
    qpath.qp_anneal_batch(handles, R, sc, seed, st, E, B, stream=torch.cuda.current_stream())
    check_fields(handles, R, sc, seed, st, E, B)


def test_batch_errors(dev):
    import torch
    h = qpath.qp_build_qubo(inputs.rect(3, 3))
    sc = qpath.schedule(10)
    n = h.info["n"]
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_batch_create([h], 2, sc, 1, [np.zeros((2, n), np.uint8)], [np.zeros(2, np.int64)])
    assert e.value.status == qpath.QP_EINVAL
    h32 = qpath.qp_build_qubo(inputs.rect(3, 3), scale=100000)  # distances beyond int16
    st = [torch.zeros((2, n), dtype=torch.uint8, device="cuda")]
    E = [torch.zeros(2, dtype=torch.int64, device="cuda")]
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_batch_create([h32], 2, sc, 1, st, E)
    assert e.value.status == qpath.QP_ERANGE


@pytest.mark.slow
def test_batch_full_256_fields(dev, orc):
    """256 fields (sides 4..16, 0-20% obstacles, irregular boundaries), 128
    replicas each, 2000 sweeps, one graph launch; every field against its own
    single-field anneal and sampled (field, replica) pairs against the oracle."""
    import torch
    fields = inputs.batch(256, seed=2026)
    handles = [qpath.qp_build_qubo(f) for f in fields]
    R, seed = 128, 1
    sc = qpath.schedule(2000)
    st, E, B = outputs(handles, R)
    b = qpath.qp_batch_create(handles, R, sc, seed, st, E, B)
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_fields(handles, R, sc, seed, st, E, B, fields=range(0, 256, 17))
    for f, rs in [(3, [0, 127]), (100, [5]), (255, [64])]:
        fl = fields[f]
        P = orc.Problem(fl.rows, fl.cols, fl.free_mask, fl.start)
        ref = orc.anneal_structured(P, rs, 2000, seed=seed + f)
        assert (st[f].cpu().numpy()[rs] == ref.states).all()
        assert (E[f].cpu().numpy()[rs] == ref.energies).all()
        assert (B[f].cpu().numpy()[rs] == ref.best).all()


def test_autotuner_picks_valid_configs_and_caches(dev, tmp_path, monkeypatch):
    import json

    import torch

    from paper_2608_25376_gb300 import autotune
    monkeypatch.setenv("QPATH_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    h = qpath.qp_build_qubo(inputs.obstacles(8, 8, 0.1, seed=1))
    w = autotune.tune_single(h, 64, 200, candidates=(1, 4, 8), window=10)
    assert w in (1, 4, 8)
    assert autotune.tune_single(h, 64, 200) == w  # from the cache
    fields = inputs.batch(8, seed=4)
    hs = [qpath.qp_build_qubo(f) for f in fields]
    wb, ctas, flags = autotune.tune_batch(hs, 8, 100, candidates_w=(2, 8), cta_factors=(0, 1), window=10)
    assert flags in (0, qpath.QP_BATCH_D_SHARED)
    d = json.load(open(tmp_path / "tune.json"))
    assert len(d) == 2
    # both stagings were timed
    e = [v for k, v in d.items() if "|batch|" in k][0]
    assert any(k.endswith(",0") for k in e["ms"]) and any(k.endswith(f",{qpath.QP_BATCH_D_SHARED}") for k in e["ms"])
    # the tuned batch gives the per-field results
    sc = qpath.schedule(100)
    st, E, B = outputs(hs, 8)
    b = qpath.qp_batch_create(hs, 8, sc, 4, st, E, B, replicas_per_cta=wb, ctas=ctas, flags=flags)
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_fields(hs, 8, sc, 4, st, E, B)


@pytest.mark.parametrize("W", [1, 3, 8])
def test_batch_with_d_staged_in_shared_memory(dev, W):
    """QP_BATCH_D_SHARED: CTAs of W replicas of one field against its d in
    shared memory (replica blocks that do not divide R included) give the
    per-field results; fields up to 300 cells."""
    import torch
    fields = inputs.batch(12, seed=9) + [inputs.obstacles(18, 18, 0.1, seed=8, start=5)]
    hs = [qpath.qp_build_qubo(f) for f in fields]
    R, seed = 10, 5
    sc = qpath.schedule(60)
    st, E, B = outputs(hs, R)
    b = qpath.qp_batch_create(hs, R, sc, seed, st, E, B, replicas_per_cta=W, ctas=7,
                              flags=qpath.QP_BATCH_D_SHARED)
    assert 1 <= b.info["replicas_per_cta"] <= W  # fewer when the largest field leaves no room
    b.run(torch.cuda.current_stream())
    torch.cuda.synchronize()
    check_fields(hs, R, sc, seed, st, E, B)
    with pytest.raises(qpath.QpError):
        qpath.qp_batch_create(hs, R, sc, seed, st, E, B, flags=8)
