"""The warm-start MLP on the GPU (tcgen05 GEMMs) against the CPU reference:
logits within 2e-2 max-abs, gradients element by element within the bf16
tolerance of tests/ws_bounds.py (the training pass is also checked tensor by
tensor on the GPU's own operands in test_gpu_ws_train.py)."""
import numpy as np
import pytest

from conftest import has_gpu
from oracle import mlp_ref
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath
from ws_bounds import grad_error_bound

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    qpath.lib()


def field_batch(n, seed):
    """Features, labels (a serpentine-like order) and steps of n synthetic fields."""
    fs = inputs.batch(n, seed=seed, lo=4, hi=12)
    X, Y, T = [], [], []
    for f in fs:
        x = qpath.qp_ws_features(f)
        C = x.shape[0]
        X.append(x)
        T.append(np.full(C, C, np.int32))
        Y.append(np.argsort(np.argsort(x[:, 1] * 16 + x[:, 0])).astype(np.int32))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(T)


def test_forward_logits_match_cpu(dev):
    m = qpath.WarmStartModel(seed=5)
    params = qpath.qp_ws_get_params(m)
    X, _, _ = field_batch(5, seed=1)
    X = X[:300]                                   # ragged: 300 rows, tiles of 128
    got = qpath.qp_ws_forward(m, X)
    ref, _ = mlp_ref.forward(params, X, bf16_storage=True)
    err = np.abs(got - ref).max()
    assert err <= 2e-2, err
    assert np.abs(ref).max() > 0.1                # not a vacuous comparison


def test_gradients_match_cpu(dev):
    m = qpath.WarmStartModel(seed=6)
    params = qpath.qp_ws_get_params(m)
    X, Y, T = field_batch(8, seed=2)
    Y[::7] = -1                                   # ignored rows
    loss, g = qpath.qp_ws_grads(m, X, Y, T)
    ref_loss, ref_g = mlp_ref.loss_and_grads(params, X, Y, T, bf16_storage=True)
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss)
    tol = grad_error_bound(params, X, Y, T)
    bad = np.abs(g - ref_g) > tol
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])
    # and against the exact float64 network, looser (bf16 storage in between)
    _, g64 = mlp_ref.loss_and_grads(params, X, Y, T, bf16_storage=False)
    rel = np.linalg.norm(g - g64) / np.linalg.norm(g64)
    assert rel <= 5e-2, rel


def test_large_batch_split_k(dev):
    """8960 rows: 70 row tiles forward, 17-way split-K for the weight gradients."""
    m = qpath.WarmStartModel(seed=7)
    params = qpath.qp_ws_get_params(m)
    X, Y, T = field_batch(140, seed=3)
    X, Y, T = X[:8960], Y[:8960], T[:8960]
    got = qpath.qp_ws_forward(m, X)
    rows = np.random.default_rng(0).choice(len(X), 400, replace=False)
    ref, _ = mlp_ref.forward(params, X[rows], bf16_storage=True)
    assert np.abs(got[rows] - ref).max() <= 2e-2
    loss, g = qpath.qp_ws_grads(m, X, Y, T)
    ref_loss, ref_g = mlp_ref.loss_and_grads(params, X, Y, T, bf16_storage=True)
    assert not (np.abs(g - ref_g) > grad_error_bound(params, X, Y, T)).any()


def test_training_reduces_loss(dev):
    m = qpath.WarmStartModel(seed=8)
    X, Y, T = field_batch(40, seed=4)
    first = qpath.qp_ws_train_step(m, X, Y, T, 1e-3)
    for _ in range(80):
        last = qpath.qp_ws_train_step(m, X, Y, T, 1e-3)
    assert last < 0.6 * first, (first, last)
    # the updated weights still give CPU-matching logits
    params = qpath.qp_ws_get_params(m)
    got = qpath.qp_ws_forward(m, X[:256])
    ref, _ = mlp_ref.forward(params, X[:256], bf16_storage=True)
    assert np.abs(got - ref).max() <= 2e-2 * max(1.0, np.abs(ref).max() / 10)


def test_infer_equals_the_three_steps(dev):
    """qp_ws_infer = features, forward and decode, for both decoders; the seed
    is a feasible one-hot state with the start cell at step 0."""
    m = qpath.WarmStartModel(seed=5)
    f = inputs.obstacles(9, 11, 0.15, seed=4, start=7)
    h = qpath.qp_build_qubo(f)
    C = h.info["C"]
    d = qpath.qp_export_dist(h)
    L = qpath.qp_ws_forward(m, qpath.qp_ws_features(f))
    start = int(np.cumsum(f.free_mask)[f.start] - 1)
    for dd, ref in ((d, qpath.qp_ws_decode_walk(L, C, start, d)), (None, qpath.qp_ws_decode(L, C, start))):
        st, path = qpath.qp_ws_infer(m, f, dd)
        assert (st == ref[0]).all() and (path == ref[1]).all()
        assert path[0] == start and sorted(path.tolist()) == list(range(C))
        assert qpath.qp_decode_path(h, st) is not None


def test_fused_forward_equals_layered(dev):
    """The one-launch forward (activations kept in shared memory) and the
    per-layer GEMM launches issue the same MMAs in the same order: the logits
    are bit-identical, on ragged sizes and after training has moved the
    weights away from their initial scale.  The gradients, computed from the
    hidden activations either mode stores, agree up to the order of the
    backward pass's fp32 atomic sums."""
    m = qpath.WarmStartModel(seed=9)
    X, Y, T = field_batch(140, seed=5)
    for _ in range(3):
        qpath.qp_ws_train_step(m, X[:4096], Y[:4096], T[:4096], 1e-3)
    for M in (1, 127, 300, 8960):
        out = {}
        for mode in (qpath.QP_WS_FORWARD_FUSED, qpath.QP_WS_FORWARD_LAYERED):
            qpath.qp_ws_set_forward_mode(m, mode)
            out[mode] = (qpath.qp_ws_forward(m, X[:M]), qpath.qp_ws_grads(m, X[:M], Y[:M], T[:M]))
        (za, (la, ga)), (zb, (lb, gb)) = out[qpath.QP_WS_FORWARD_FUSED], out[qpath.QP_WS_FORWARD_LAYERED]
        assert np.array_equal(za, zb), (M, np.abs(za - zb).max())
        assert abs(la - lb) <= 1e-6 * abs(lb), (M, la, lb)
        assert np.linalg.norm(ga - gb) <= 1e-5 * np.linalg.norm(gb), M
    qpath.qp_ws_set_forward_mode(m, qpath.QP_WS_FORWARD_FUSED)
    with pytest.raises(qpath.QpError):
        qpath.qp_ws_set_forward_mode(m, 2)


def test_training_repeats_bit_for_bit(dev):
    """Every sum over rows in a training step is taken in a fixed order, so two
    models from the same seed trained on the same batches end with the same
    weights, moments and losses, bit for bit (split-K included: 8960 rows)."""
    X, Y, T = field_batch(140, seed=9)
    X, Y, T = X[:8960], Y[:8960], T[:8960]
    runs = []
    for _ in range(2):
        m = qpath.WarmStartModel(seed=21)
        losses = [qpath.qp_ws_train_step(m, X, Y, T, 1e-3) for _ in range(3)]
        runs.append((losses, qpath.qp_ws_get_params(m)))
    assert runs[0][0] == runs[1][0]
    assert np.array_equal(runs[0][1].view(np.uint32), runs[1][1].view(np.uint32))
