"""The warm-start network's training pass on the GPU, element by element.

1. Every tensor a pass stores is checked against the CPU reference evaluated on
   the GPU's own operands (read back with qp_ws_get_buffer): the bf16 weight
   copies and their transposes (bit-exact roundings of the fp32 masters), the
   bf16 inputs (bit-exact), each hidden activation and back-propagated
   gradient (within half a bf16 ulp of the float64 value plus the fp32
   summation bound), the fp32 logits and every weight and bias gradient
   (within the fp32 summation bound: n 2^-24 of the sum of |terms|, doubled).
2. The gradients against the independent CPU reference, element-wise within
   the bf16 tolerance of tests/ws_bounds.py.
3. Adam: after one, two and three qp_ws_train_step calls, the fp32 masters,
   both moments, the bf16 weights and their transposes against the reference
   Adam step (Kingma & Ba) applied to the gradients the GPU used.
"""
import numpy as np
import pytest

from conftest import has_gpu
from oracle import mlp_ref
from paper_2608_25376_gb300 import build as qbuild
from paper_2608_25376_gb300 import inputs, qpath
from ws_bounds import U_F32, bf16_bits, grad_error_bound, ulp_bf16

pytestmark = pytest.mark.gpu

f64 = qpath.bf16_bits_to_float


@pytest.fixture(scope="module")
def dev():
    if not has_gpu():
        pytest.skip("no CUDA device")
    qbuild.build()
    qpath.lib()


def field_batch(n, seed):
    fs = inputs.batch(n, seed=seed, lo=4, hi=12)
    X, Y, T = [], [], []
    for f in fs:
        x = qpath.qp_ws_features(f)
        C = x.shape[0]
        X.append(x)
        T.append(np.full(C, C, np.int32))
        Y.append(np.argsort(np.argsort(x[:, 1] * 16 + x[:, 0])).astype(np.int32))
    return np.concatenate(X), np.concatenate(Y), np.concatenate(T)


def offsets():
    return np.cumsum([0] + [x for (no, ni) in mlp_ref.DIMS for x in (no * ni, no)])


def split(flat):
    o = offsets()
    return [(flat[o[2 * l]:o[2 * l + 1]].reshape(mlp_ref.DIMS[l]), flat[o[2 * l + 1]:o[2 * l + 2]])
            for l in range(4)]


def check_stored_bf16(got_bits, ref, absum, n_terms, what):
    """A bf16 element the GPU rounded from an fp32 sum: within half an ulp of
    the float64 value plus the summation bound."""
    got = f64(got_bits)
    acc = 2 * (n_terms + 16) * U_F32 * absum
    tol = 0.5 * ulp_bf16(np.maximum(np.abs(got), np.abs(ref))) + acc
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (what, int(bad.sum()), np.argwhere(bad)[:5])
    return float((got_bits == bf16_bits(ref)).mean())


def check_fp32_sum(got, ref, absum, n_terms, what):
    tol = 2 * (n_terms + 16) * U_F32 * absum + 1e-30
    bad = np.abs(np.asarray(got, np.float64) - ref) > tol
    assert not bad.any(), (what, int(bad.sum()), np.argwhere(bad)[:5])


def check_pass_on_gpu_operands(m, X, Y, T):
    """One qp_ws_grads pass; every stored tensor against its operands."""
    M = len(X)
    _, g = qpath.qp_ws_grads(m, X, Y, T)
    params = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_PARAMS)
    assert np.array_equal(g, qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_GRADS))
    layers = split(params)
    grads = split(g)
    wq_bits = [qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_W_BF16 + l) for l in range(4)]
    for l in range(4):
        assert np.array_equal(wq_bits[l], bf16_bits(layers[l][0])), l
        assert np.array_equal(qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_WT_BF16 + l), wq_bits[l].T), l
    Wq = [f64(b) for b in wq_bits]
    x0 = qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_X0, M)
    assert np.array_equal(x0, bf16_bits(X))
    acts_bits = [x0] + [qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_H1 + l, M) for l in range(3)]
    acts = [f64(a) for a in acts_bits]
    exact = []
    for l in range(3):
        b = layers[l][1]
        ref = mlp_ref.layer_forward(acts[l], Wq[l], b, relu=True)
        absum = np.abs(acts[l]) @ np.abs(Wq[l]).T + np.abs(b)
        exact.append(check_stored_bf16(acts_bits[l + 1], ref, absum, acts[l].shape[1] + 1, f"H{l + 1}"))
    Z = qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_Z, M)
    b3 = layers[3][1]
    check_fp32_sum(Z, mlp_ref.layer_forward(acts[3], Wq[3], b3, relu=False),
                   np.abs(acts[3]) @ np.abs(Wq[3]).T + np.abs(b3), 257, "Z")
    # dZ from the GPU's logits: fp32 exp, sum and divide, then bf16
    dz_bits = qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_DZ, M)
    ref = mlp_ref.ce_grad(Z.astype(np.float64), Y, T, M)
    dz = f64(dz_bits)
    tol = 0.5 * ulp_bf16(np.maximum(np.abs(dz), np.abs(ref))) + 1e-5 * np.abs(ref) + 1e-7 / M
    assert not (np.abs(dz - ref) > tol).any(), "dZ"
    dys = [f64(qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_DH1 + l, M)) for l in range(3)] + [dz]
    dys_bits = [qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_DH1 + l, M) for l in range(3)] + [dz_bits]
    for l in range(3, -1, -1):
        dY, Xl = dys[l], acts[l]
        dW, db, dX = mlp_ref.layer_backward(dY, Xl, Wq[l], Xl if l > 0 else None)
        check_fp32_sum(grads[l][0], dW, np.abs(dY).T @ np.abs(Xl), M, f"dW{l}")
        check_fp32_sum(grads[l][1], db, np.abs(dY).sum(axis=0), M, f"db{l}")
        if l > 0:
            absum = np.abs(dY) @ np.abs(Wq[l])
            exact.append(check_stored_bf16(dys_bits[l - 1], dX, absum, Wq[l].shape[0], f"dH{l}"))
    return g, params, exact


def test_training_pass_elementwise_on_gpu_operands(dev):
    m = qpath.WarmStartModel(seed=6)
    X, Y, T = field_batch(8, seed=2)
    Y[::7] = -1                                   # ignored rows
    _, _, exact = check_pass_on_gpu_operands(m, X, Y, T)
    # a rounding boundary between the fp32 and float64 sums is rare
    assert min(exact) > 0.99, exact


def test_training_pass_elementwise_split_k(dev):
    """8960 rows: 70 row tiles, 17-way split-K with fp32 atomics for dW."""
    m = qpath.WarmStartModel(seed=7)
    X, Y, T = field_batch(140, seed=3)
    check_pass_on_gpu_operands(m, X[:8960], Y[:8960], T[:8960])


@pytest.mark.parametrize("seed,n_fields", [(2, 8), (3, 60)])
def test_gradients_elementwise_against_cpu_reference(dev, seed, n_fields):
    m = qpath.WarmStartModel(seed=6)
    params = qpath.qp_ws_get_params(m)
    X, Y, T = field_batch(n_fields, seed=seed)
    Y[::7] = -1
    loss, g = qpath.qp_ws_grads(m, X, Y, T)
    ref_loss, ref_g = mlp_ref.loss_and_grads(params, X, Y, T, bf16_storage=True)
    assert abs(loss - ref_loss) <= 1e-3 * abs(ref_loss)
    tol = grad_error_bound(params, X, Y, T)
    bad = np.abs(g - ref_g) > tol
    assert not bad.any(), (int(bad.sum()), np.argwhere(bad)[:5])


def test_adam_steps_match_reference(dev):
    m = qpath.WarmStartModel(seed=4)
    X, Y, T = field_batch(10, seed=7)
    lr = np.float32(2e-3)
    b1, b2, eps = float(np.float32(0.9)), float(np.float32(0.999)), float(np.float32(1e-8))
    w = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_PARAMS).astype(np.float64)
    mo = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_ADAM_M).astype(np.float64)
    vo = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_ADAM_V).astype(np.float64)
    assert not mo.any() and not vo.any()
    for t in (1, 2, 3):
        qpath.qp_ws_train_step(m, X, Y, T, float(lr))
        g = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_GRADS).astype(np.float64)
        w_ref, m_ref, v_ref = mlp_ref.adam_step(w, mo, vo, g, t, float(lr), b1, b2, eps)
        w_gpu = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_PARAMS).astype(np.float64)
        m_gpu = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_ADAM_M).astype(np.float64)
        v_gpu = qpath.qp_ws_get_state(m, qpath.QP_WS_STATE_ADAM_V).astype(np.float64)
        # fp32 arithmetic: a few units of 2^-24 of the terms of each sum
        tol_m = 4 * U_F32 * (b1 * np.abs(mo) + (1 - b1) * np.abs(g)) + 1e-44
        tol_v = 4 * U_F32 * (b2 * vo + (1 - b2) * g * g) + 1e-44
        assert not (np.abs(m_gpu - m_ref) > tol_m).any(), ("m", t)
        assert not (np.abs(v_gpu - v_ref) > tol_v).any(), ("v", t)
        # the update: fp32 powf for the bias corrections (1 - 0.999^t cancels
        # to a few parts in 1e5 at small t), sqrtf and divides
        upd = np.abs(w - w_ref)
        tol_w = U_F32 * np.abs(w_ref) + 5e-5 * upd + 1e-30
        assert not (np.abs(w_gpu - w_ref) > tol_w).any(), ("w", t)
        assert upd.max() > 0.5 * float(lr)      # the step did move the weights
        for l, (W, _) in enumerate(split(w_gpu)):
            wb = qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_W_BF16 + l)
            assert np.array_equal(wb, bf16_bits(W)), ("bf16", l, t)
            assert np.array_equal(qpath.qp_ws_get_buffer(m, qpath.QP_WS_BUF_WT_BF16 + l), wb.T), ("bf16^T", l, t)
        w, mo, vo = w_gpu, m_gpu, v_gpu
