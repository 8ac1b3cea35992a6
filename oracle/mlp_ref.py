"""CPU reference of the warm-start MLP -- TEST INFRASTRUCTURE.

Plain numpy, written from the definition of the network (16 -> 256 -> 256 ->
256 -> 256, ReLU after the first three layers, softmax cross-entropy over the
steps t < C of each cell's field) and of back-propagation.  Products are summed
in float64.  With ``bf16=True`` every tensor the GPU stores in bfloat16 (inputs,
weights, hidden activations, the back-propagated gradients dZ and dH) is
rounded to bfloat16 (round half to even) at the same places, so the GPU can be
compared within accumulation-order differences; with ``bf16=False`` it is the
exact float64 network used to pin the backward pass by finite differences.
Also: one layer at a time (forward, the cross-entropy gradient, backward) on
explicit inputs, so each GPU product can be checked on the GPU's own stored
operands; the Adam update (Kingma & Ba, ICLR 2015, Algorithm 1); and the
decodes of step logits into a path.
"""
from __future__ import annotations

import numpy as np

DIMS = [(256, 16), (256, 256), (256, 256), (256, 256)]  # (out, in) per layer


def bf16(x):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    a = np.ascontiguousarray(x, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def unflatten(params):
    out, o = [], 0
    for (no, ni) in DIMS:
        W = params[o:o + no * ni].reshape(no, ni).astype(np.float64)
        o += no * ni
        b = params[o:o + no].astype(np.float64)
        o += no
        out.append((W, b))
    return out


def flatten(grads):
    return np.concatenate([np.concatenate([gW.reshape(-1), gb]) for gW, gb in grads])


def forward(params, feats, bf16_storage=True):
    """-> (logits [M, 256], activations list [X0, H1, H2, H3])"""
    q = bf16 if bf16_storage else (lambda v: np.asarray(v, np.float64))
    layers = unflatten(params)
    X = q(feats)
    acts = [X]
    for l, (W, b) in enumerate(layers):
        A = X @ q(W).T + b
        if l < 3:
            X = q(np.maximum(A, 0.0))
            acts.append(X)
        else:
            return A, acts
    raise AssertionError


def loss_and_grads(params, feats, labels, steps, bf16_storage=True):
    """Mean cross-entropy over cells with label >= 0 and its gradient (flat, in
    the parameter layout)."""
    q = bf16 if bf16_storage else (lambda v: np.asarray(v, np.float64))
    layers = unflatten(params)
    Z, acts = forward(params, feats, bf16_storage)
    M = len(labels)
    T = Z.shape[1]
    mask = np.arange(T)[None, :] < np.asarray(steps)[:, None]
    valid = np.asarray(labels) >= 0
    Zm = np.where(mask, Z, -np.inf)
    Zm = Zm - Zm.max(axis=1, keepdims=True)
    P = np.where(mask, np.exp(Zm), 0.0)
    P /= P.sum(axis=1, keepdims=True)
    lab = np.where(valid, labels, 0)
    loss = -np.log(np.maximum(P[np.arange(M), lab], 1e-300))[valid].sum() / M
    Y = np.zeros_like(P)
    Y[np.arange(M), lab] = 1.0
    dZ = np.where(valid[:, None], (P - Y) / M, 0.0)
    dY = q(dZ)
    grads = [None] * 4
    for l in range(3, -1, -1):
        W, _ = layers[l]
        X = acts[l]
        grads[l] = (dY.T @ X, dY.sum(axis=0))
        if l == 0:
            break
        dX = dY @ q(W)
        dY = q(np.where(X > 0, dX, 0.0))
    return loss, flatten(grads)


def layer_forward(X, Wq, b, relu):
    """One layer on given operands, summed in float64: A = X Wq^T + b, then
    ReLU when relu (no rounding: the caller rounds what is stored)."""
    A = np.asarray(X, np.float64) @ np.asarray(Wq, np.float64).T + np.asarray(b, np.float64)
    return np.maximum(A, 0.0) if relu else A


def ce_grad(Z, labels, steps, M):
    """Gradient of the mean softmax cross-entropy with respect to the logits Z
    (rows with label < 0 contribute nothing; logits t >= steps are masked; M is
    the divisor of the mean), in float64."""
    Z = np.asarray(Z, np.float64)
    T = Z.shape[1]
    mask = np.arange(T)[None, :] < np.asarray(steps)[:, None]
    valid = np.asarray(labels) >= 0
    Zm = np.where(mask, Z, -np.inf)
    Zm = Zm - Zm.max(axis=1, keepdims=True)
    P = np.where(mask, np.exp(Zm), 0.0)
    P /= P.sum(axis=1, keepdims=True)
    lab = np.where(valid, labels, 0)
    Y = np.zeros_like(P)
    Y[np.arange(len(lab)), lab] = 1.0
    return np.where(valid[:, None], (P - Y) / M, 0.0)


def layer_backward(dY, X, Wq, relu_ref):
    """Back-propagation through one layer on given operands, float64:
    dW = dY^T X, db = column sums of dY, and (when relu_ref is given) the
    gradient at the layer's input, dY Wq, zeroed where relu_ref <= 0."""
    dY = np.asarray(dY, np.float64)
    dW = dY.T @ np.asarray(X, np.float64)
    db = dY.sum(axis=0)
    dX = None
    if relu_ref is not None:
        dX = np.where(np.asarray(relu_ref) > 0, dY @ np.asarray(Wq, np.float64), 0.0)
    return dW, db, dX


def adam_step(w, m, v, g, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, "Adam: A Method for Stochastic
    Optimization", ICLR 2015, Algorithm 1) in float64, t counting from 1:
        m_t = b1 m_{t-1} + (1 - b1) g,   v_t = b2 v_{t-1} + (1 - b2) g^2,
        w_t = w_{t-1} - lr (m_t / (1 - b1^t)) / (sqrt(v_t / (1 - b2^t)) + eps).
    -> (w_t, m_t, v_t)"""
    w, m, v, g = (np.asarray(a, np.float64) for a in (w, m, v, g))
    m_t = b1 * m + (1.0 - b1) * g
    v_t = b2 * v + (1.0 - b2) * g * g
    m_hat = m_t / (1.0 - b1 ** t)
    v_hat = v_t / (1.0 - b2 ** t)
    return w - lr * m_hat / (np.sqrt(v_hat) + eps), m_t, v_t


def greedy_decode(logits, C, start_cell):
    """Step 0 is the start cell; then the largest logit over unassigned cells
    and free steps 1..C-1 fixes one (cell, step) pair at a time; ties go to the
    smaller cell, then the smaller step."""
    L = np.asarray(logits, dtype=np.float64)[:C, :C]
    path = [-1] * C
    path[0] = start_cell
    cells = set(range(C)) - {start_cell}
    steps = set(range(1, C))
    while cells:
        best = None
        for i in sorted(cells):
            for t in sorted(steps):
                v = L[i, t]
                if best is None or v > best[0]:
                    best = (v, i, t)
        _, i, t = best
        path[t] = i
        cells.remove(i)
        steps.remove(t)
    return path


def walk_decode(logits, C, start_cell, d):
    """From the start cell, step to the nearest unvisited cell; ties by the
    smaller expected step under softmax over t < C, then the smaller cell."""
    L = np.asarray(logits, dtype=np.float64)[:C, :C]
    e = []
    for i in range(C):
        z = L[i] - L[i].max()
        p = np.exp(z)
        e.append(float((p * np.arange(C)).sum() / p.sum()))
    path, seen, cur = [start_cell], {start_cell}, start_cell
    for _ in range(1, C):
        cands = [j for j in range(C) if j not in seen]
        nxt = min(cands, key=lambda j: (int(d[cur][j]), e[j], j))
        path.append(nxt)
        seen.add(nxt)
        cur = nxt
    return path


def expected_steps(logits, steps):
    """E_m = sum_{t < T_m} t softmax(z_m)_t over the first T_m = steps[m]
    logits of each row, in float64."""
    Z = np.asarray(logits, np.float64)
    out = np.empty(len(Z))
    for m, T in enumerate(np.asarray(steps)):
        z = Z[m, :T] - Z[m, :T].max()
        p = np.exp(z)
        out[m] = float((p * np.arange(T)).sum() / p.sum())
    return out


def walk(d, C, start_cell, score=None, slack=0):
    """The walk decode, step by step: from the start cell, each step goes to an
    unvisited cell j with d(cur, j) <= (nearest unvisited distance) + slack,
    choosing the smallest (score[j], d(cur, j), j), or the smallest
    (d(cur, j), j) without a score.  Scores compare as real numbers."""
    path, seen, cur = [start_cell], {start_cell}, start_cell
    for _ in range(1, C):
        cands = [j for j in range(C) if j not in seen]
        dmin = min(int(d[cur][j]) for j in cands)
        near = [j for j in cands if int(d[cur][j]) <= dmin + slack]
        if score is None:
            nxt = min(near, key=lambda j: (int(d[cur][j]), j))
        else:
            nxt = min(near, key=lambda j: (float(score[j]), int(d[cur][j]), j))
        path.append(nxt)
        seen.add(nxt)
        cur = nxt
    return path
