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


def test_adam_reference_matches_torch_optimizer():
    """The reference Adam step equals torch.optim.Adam (an independent library
    implementation of Kingma & Ba's algorithm) in float64 over three steps."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    w0 = rng.normal(0, 1, 50)
    grads = [rng.normal(0, 1e-2, 50) * rng.random(50) for _ in range(3)]
    p = torch.tensor(w0.copy(), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=3e-3, betas=(0.9, 0.999), eps=1e-8)
    w, m, v = w0.copy(), np.zeros(50), np.zeros(50)
    for t, g in enumerate(grads, start=1):
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        w, m, v = mlp_ref.adam_step(w, m, v, g, t, 3e-3)
        st = opt.state[p]
        assert np.abs(p.detach().numpy() - w).max() <= 1e-15
        assert np.abs(st["exp_avg"].numpy() - m).max() <= 1e-18
        assert np.abs(st["exp_avg_sq"].numpy() - v).max() <= 1e-20


def test_adam_reference_constant_gradient_closed_form():
    """With the same gradient g at every step the bias corrections make
    m_hat = g and v_hat = g^2 exactly, so each step moves w by lr g / (|g| + eps)
    (a dropped correction moves it by about 3 lr instead of lr at step 1)."""
    g = np.array([0.5, -2.0, 1e-3, -7e-6])
    w, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    lr = 1e-2
    for t in range(1, 6):
        w1, m, v = mlp_ref.adam_step(w, m, v, g, t, lr)
        np.testing.assert_allclose(w - w1, lr * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
        w = w1


def test_layer_functions_compose_to_the_reference_gradients():
    """Forward, cross-entropy gradient and backward one layer at a time, with
    bf16 rounding where the network stores a tensor, give loss_and_grads."""
    params, feats, labels, steps = _small_problem(3)
    q = mlp_ref.bf16
    layers = mlp_ref.unflatten(params)
    X = [q(feats)]
    for l, (W, b) in enumerate(layers[:3]):
        X.append(q(mlp_ref.layer_forward(X[-1], q(W), b, relu=True)))
    Z = mlp_ref.layer_forward(X[3], q(layers[3][0]), layers[3][1], relu=False)
    Zr, _ = mlp_ref.forward(params, feats, bf16_storage=True)
    assert np.array_equal(Z, Zr)
    dY = q(mlp_ref.ce_grad(Z, labels, steps, len(labels)))
    grads = [None] * 4
    for l in range(3, -1, -1):
        dW, db, dX = mlp_ref.layer_backward(dY, X[l], q(layers[l][0]), X[l] if l > 0 else None)
        grads[l] = (dW, db)
        if l > 0:
            dY = q(dX)
    _, g = mlp_ref.loss_and_grads(params, feats, labels, steps, bf16_storage=True)
    assert np.array_equal(mlp_ref.flatten(grads), g)


def _grid_d(rows, cols, mask=None):
    """Exact distances round(100 * euclid) between the free cells, row-major."""
    import math
    cells = [(r, c) for r in range(rows) for c in range(cols) if mask is None or mask[r * cols + c]]
    C = len(cells)
    d = [[0] * C for _ in range(C)]
    for a, (r0, c0) in enumerate(cells):
        for b, (r1, c1) in enumerate(cells):
            q = 10000 * ((r0 - r1) ** 2 + (c0 - c1) ** 2)
            s = math.isqrt(q)
            d[a][b] = s + (1 if q - s * s > s else 0)
    return d, cells


def test_walk_reference_plain_walk_is_the_serpentine():
    """On an obstacle-free rectangle from a corner, the nearest-cell walk with
    ties to the smaller cell id goes along each row and back: the
    boustrophedon, whose length 100 (C - 1) is the optimum."""
    for rows, cols in ((3, 3), (3, 5), (4, 4), (5, 2)):
        d, cells = _grid_d(rows, cols)
        C = len(cells)
        path = mlp_ref.walk(d, C, 0)
        serp = [r * cols + (c if r % 2 == 0 else cols - 1 - c) for r in range(rows) for c in range(cols)]
        assert path == serp
        assert sum(d[path[t]][path[t + 1]] for t in range(C - 1)) == 100 * (C - 1)


def test_walk_reference_follows_the_score_within_the_slack():
    """With an unlimited slack the score alone orders the walk: the score of an
    optimal path's step order (brute force over permutations, start fixed)
    gives back that path and its optimal length; a constant score gives the
    plain walk; slack 0 keeps every step at the nearest distance."""
    import itertools
    mask = [1, 1, 0, 1, 1, 1, 1, 0, 1]  # 3 x 3 with two obstacles: 7 cells
    d, cells = _grid_d(3, 3, mask)
    C = len(cells)
    best = min(itertools.permutations(range(1, C)),
               key=lambda p: sum(d[a][b] for a, b in zip((0,) + p, p)))
    opt = [0] + list(best)
    opt_len = sum(d[a][b] for a, b in zip(opt, opt[1:]))
    score = [0.0] * C
    for t, i in enumerate(opt):
        score[i] = float(t)
    path = mlp_ref.walk(d, C, 0, score, slack=10 ** 9)
    assert path == opt and sum(d[a][b] for a, b in zip(path, path[1:])) == opt_len
    assert mlp_ref.walk(d, C, 0, [3.5] * C, slack=150) == mlp_ref.walk(d, C, 0, None, slack=150)
    p0 = mlp_ref.walk(d, C, 0, score, slack=0)
    for t in range(1, C):
        rest = [j for j in range(C) if j not in p0[:t]]
        assert d[p0[t - 1]][p0[t]] == min(d[p0[t - 1]][j] for j in rest)
    assert sorted(p0) == list(range(C)) and p0[0] == 0


def test_expected_steps_reference_closed_forms():
    """Uniform logits over T steps: E = (T - 1) / 2; one dominant logit at k: E = k."""
    Z = np.zeros((3, 256))
    Z[2, 17] = 800.0
    E = mlp_ref.expected_steps(Z, [1, 40, 90])
    assert E[0] == 0.0 and abs(E[1] - 19.5) < 1e-12 and abs(E[2] - 17.0) < 1e-12


@pytest.mark.parametrize("logits,start,path", [
    # the two largest free entries tie (5 at step 1 for cells 0 and 2): the smaller cell takes step 1
    ([[0, 5, 1], [9, 9, 9], [0, 5, 2]], 1, [1, 0, 2]),
    # the largest entry (7) fixes cell 0 at step 2 first; cell 2 then takes step 1 although 6 < 7
    ([[0, 1, 7], [9, 9, 9], [0, 6, 3]], 1, [1, 2, 0]),
    # within one cell, equal logits go to the smaller step; the start's row and step 0 never count
    ([[9, 9, 9, 9], [0, 4, 4, 4], [0, 1, 2, 3], [99, 0, 0, 1]], 0, [0, 1, 3, 2]),
])
def test_greedy_decode_hand_worked(logits, start, path):
    """Pins of the plain greedy matching, worked by hand from its definition."""
    L = np.asarray(logits, np.float32)
    assert mlp_ref.greedy_decode(L, L.shape[0], start) == path
