"""The device decode of the warm start against its CPU reference: expected
steps within fp32 rounding of the float64 values, and the walk (with and
without a score, several slacks) path for path, given the same scores."""
import numpy as np
import pytest

from conftest import has_gpu
from oracle import mlp_ref
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    qpath.lib()


def test_expected_steps_match_reference(dev):
    import torch
    rng = np.random.default_rng(5)
    m = qpath.WarmStartModel(seed=3)
    fields = inputs.batch(6, seed=12, lo=4, hi=16)
    X = np.concatenate([qpath.qp_ws_features(f) for f in fields])
    steps = np.concatenate([np.full(f.n_cells, f.n_cells, np.int32) for f in fields])
    Z = np.concatenate([qpath.qp_ws_forward(m, X), rng.normal(0, 4, (300, 256)).astype(np.float32)])
    steps = np.concatenate([steps, rng.integers(1, 257, 300).astype(np.int32)])
    Zd = torch.from_numpy(Z).cuda()
    Sd = torch.from_numpy(steps).cuda()
    E = qpath.qp_ws_expected_steps(Zd, Sd).cpu().numpy()
    ref = mlp_ref.expected_steps(Z, steps)
    assert np.abs(E - ref).max() <= 1e-4 + 1e-4 * ref.max()
    assert (E[steps == 1] == 0).all()


def _check_walk(h, f, score, slack):
    import torch
    C = h.info["C"]
    d = qpath.qp_export_dist(h)
    start = int(np.cumsum(f.free_mask)[f.start] - 1)
    sd = None if score is None else torch.from_numpy(np.ascontiguousarray(score, np.float32)).cuda()
    st, path, ln = qpath.qp_ws_walk(h, sd, slack)
    torch.cuda.synchronize()
    path = path.cpu().numpy()
    ref = mlp_ref.walk(d, C, start, None if score is None else np.asarray(score, np.float32), slack)
    assert path.tolist() == ref, (C, slack, score is None)
    assert int(ln.item()) == int(sum(d[a, b] for a, b in zip(ref, ref[1:])))
    x = st.cpu().numpy().reshape(C, C)
    assert (x.sum(1) == 1).all() and (x[np.arange(C), path] == 1).all()


@pytest.mark.parametrize("shape", [(4, 4, 0.0, 0), (6, 7, 0.2, 3), (16, 16, 0.15, 0), (12, 9, 0.1, 40)])
def test_walk_matches_reference(dev, shape):
    rows, cols, p, start = shape
    f = inputs.obstacles(rows, cols, p, seed=rows * cols, start=start)
    h = qpath.qp_build_qubo(f)
    C = h.info["C"]
    rng = np.random.default_rng(C)
    m = qpath.WarmStartModel(seed=2)
    E = mlp_ref.expected_steps(qpath.qp_ws_forward(m, qpath.qp_ws_features(f)), np.full(C, C))
    scores = [None, E.astype(np.float32), np.round(rng.random(C) * 4) / 2 - 1.0]  # the last with ties and negatives
    for score in scores:
        for slack in (0, 100, 141, 250, 10 ** 9):
            _check_walk(h, f, score, slack)


def test_walk_large_field_without_score(dev):
    """491 cells (the 24x24 workload): the plain nearest-cell walk."""
    f = inputs.WORKLOADS["24x24-p0.15"]["field"]()
    h = qpath.qp_build_qubo(f)
    _check_walk(h, f, None, 0)
    _check_walk(h, f, None, 100)


def test_walk_refuses_host_buffers(dev):
    f = inputs.rect(3, 3)
    h = qpath.qp_build_qubo(f)
    with pytest.raises(qpath.QpError) as e:
        qpath.qp_ws_walk(h, None, 0, np.zeros(81, np.uint8), np.zeros(9, np.int32), np.zeros(1, np.int64))
    assert e.value.status == qpath.QP_EINVAL


@pytest.mark.parametrize("C,ld,seed", [(1, 1, 0), (2, 2, 1), (7, 256, 2), (64, 64, 3), (131, 256, 4), (256, 256, 5),
                                       (200, 203, 6)])
def test_greedy_decode_on_device_matches_reference(dev, C, ld, seed):
    """qp_ws_greedy against the host decode and, up to 64 cells, the plain CPU
    restatement, path for path, on logits with ties (equal values in one row,
    across rows, and -0 against +0)."""
    import torch
    rng = np.random.default_rng(seed)
    logits = np.round(rng.normal(0, 2, size=(C, ld)), 1).astype(np.float32)  # coarse values: many ties
    if C > 4:
        logits[1, 2] = -0.0
        logits[3, 2] = 0.0
        logits[2, 1:4] = logits.max() + 1  # one row's maximum at three steps
    start = int(rng.integers(C))
    st, path = qpath.qp_ws_greedy(torch.from_numpy(logits).cuda(), C, start)
    torch.cuda.synchronize()
    path = path.cpu().numpy().tolist()
    _, host = qpath.qp_ws_decode(logits, C, start)
    assert path == host.tolist()
    if C <= 64:
        assert path == mlp_ref.greedy_decode(logits, C, start)
    x = st.cpu().numpy().reshape(C, C)
    assert (x.sum(axis=0) == 1).all() and (x.sum(axis=1) == 1).all() and x[0, start] == 1


def test_greedy_decode_refuses_bad_arguments(dev):
    import torch
    Z = torch.zeros((8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(qpath.QpError):
        qpath.qp_ws_greedy(Z, 9, 0)  # a row stride shorter than the field
    with pytest.raises(qpath.QpError):
        qpath.qp_ws_greedy(Z.cpu(), 8, 0)  # host logits
    with pytest.raises(qpath.QpError):
        qpath.qp_ws_greedy(Z, 8, 8)  # start outside the field
