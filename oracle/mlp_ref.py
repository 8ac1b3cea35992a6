"""CPU reference of the warm-start MLP -- TEST INFRASTRUCTURE.

Plain numpy, written from the definition of the network (16 -> 256 -> 256 ->
256 -> 256, ReLU after the first three layers, softmax cross-entropy over the
steps t < C of each cell's field) and of back-propagation.  Products are summed
in float64.  With ``bf16=True`` every tensor the GPU stores in bfloat16 (inputs,
weights, hidden activations, the back-propagated gradients dZ and dH) is
rounded to bfloat16 (round half to even) at the same places, so the GPU can be
compared within accumulation-order differences; with ``bf16=False`` it is the
exact float64 network used to pin the backward pass by finite differences.
Also: the greedy decode of step logits into a path.
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
