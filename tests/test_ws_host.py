"""CPU checks of the warm start: the reference back-propagation against finite
differences, the features, and the greedy decode against its plain restatement."""
import numpy as np
import pytest

from oracle import mlp_ref
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath


@pytest.fixture(scope="module")
def L():
    qbuild.build()
    return qpath.lib()


def _small_problem(seed, M=24):
    rng = np.random.default_rng(seed)
    params = np.concatenate([np.concatenate([rng.normal(0, 1.0 / np.sqrt(ni), no * ni), rng.normal(0, 0.1, no)])
                             for (no, ni) in mlp_ref.DIMS])
    feats = rng.random((M, 16))
    steps = rng.integers(5, 40, M)
    labels = np.array([rng.integers(0, s) for s in steps])
    labels[3] = -1
    return params, feats, labels, steps


def test_reference_backward_matches_finite_differences():
    params, feats, labels, steps = _small_problem(1)
    loss, g = mlp_ref.loss_and_grads(params, feats, labels, steps, bf16_storage=False)
    rng = np.random.default_rng(2)
    offs = np.cumsum([0] + [no * ni + no for (no, ni) in mlp_ref.DIMS])
    idx = np.concatenate([rng.integers(offs[l], offs[l + 1], 6) for l in range(4)])
    eps = 1e-5
    for k in idx:
        p1 = params.copy()
        p1[k] += eps
        p2 = params.copy()
        p2[k] -= eps
        fd = (mlp_ref.loss_and_grads(p1, feats, labels, steps, False)[0]
              - mlp_ref.loss_and_grads(p2, feats, labels, steps, False)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 + 1e-5 * abs(fd), (k, fd, g[k])


def test_reference_softmax_ce_closed_form():
    """Zero weights -> uniform softmax over the C valid steps: loss = mean log C."""
    params = np.zeros(sum(no * ni + no for (no, ni) in mlp_ref.DIMS))
    feats = np.random.default_rng(0).random((5, 16))
    steps = np.array([3, 7, 10, 2, 256])
    labels = np.array([0, 6, 9, 1, 100])
    loss, _ = mlp_ref.loss_and_grads(params, feats, labels, steps, False)
    assert abs(loss - np.log(steps).mean()) < 1e-12


def test_bf16_rounding_matches_definition():
    x = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 65504.0, 1e-20])
    r = mlp_ref.bf16(x)
    # bf16 has 8 significant bits: 1 + k/128
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == 1.0078125
    assert abs(r[3] - (-3.140625)) < 1e-12


def test_features_of_a_small_field(L):
    f = inputs.Field(2, 3, np.array([1, 0, 1, 1, 1, 1], np.uint8), 3)
    x = qpath.qp_ws_features(f)
    assert x.shape == (5, 16)
    # cell 0 is (0, 0); start is grid cell 3 = (1, 0)
    assert np.allclose(x[0, :2], [0.0, 0.0]) and np.allclose(x[0, 3:5], [0.0, 1 / 15])
    assert np.allclose(x[:, 7], 5 / 256) and np.allclose(x[:, 14], 1.0) and np.allclose(x[:, 15], 0.0)
    assert np.allclose(x[2, 13], 1.0)  # cell 2 = (1, 0): odd row
    # (0, 0) has neighbours (0,1) blocked, (1,0), (1,1) free and 5 outside: 6/8 blocked
    assert abs(x[0, 2] - 6 / 8) < 1e-7


@pytest.mark.parametrize("C,seed", [(1, 0), (2, 1), (7, 2), (30, 3), (64, 4)])
def test_decode_matches_plain_greedy_and_is_a_path(L, C, seed):
    rng = np.random.default_rng(seed)
    logits = rng.normal(size=(C, 256)).astype(np.float32)
    if C > 5:
        logits[2, 3] = logits[4, 3] = logits.max() + 1  # a tie, broken toward the smaller cell
    start = int(rng.integers(C))
    st, path = qpath.qp_ws_decode(logits, C, start)
    assert path.tolist() == mlp_ref.greedy_decode(logits, C, start)
    x = st.reshape(C, C)
    assert (x.sum(axis=0) == 1).all() and (x.sum(axis=1) == 1).all() and x[0, start] == 1


@pytest.mark.parametrize("shape,seed", [((3, 4), 0), ((6, 7), 1), ((9, 9), 2)])
def test_walk_decode_matches_plain_restatement(L, orc, shape, seed):
    f = inputs.obstacles(*shape, 0.15, seed=seed)
    P = orc.Problem(f.rows, f.cols, f.free_mask, f.start)
    rng = np.random.default_rng(seed)
    logits = rng.normal(size=(P.C, 256)).astype(np.float32)
    st, path = qpath.qp_ws_decode_walk(logits, P.C, P.start_cell, P.d)
    assert path.tolist() == mlp_ref.walk_decode(logits, P.C, P.start_cell, P.d)
    x = st.reshape(P.C, P.C)
    assert (x.sum(axis=0) == 1).all() and (x.sum(axis=1) == 1).all() and x[0, P.start_cell] == 1
