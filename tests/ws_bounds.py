"""Tolerances for comparing the GPU warm-start network with its CPU reference.

Both sides store the same tensors in bfloat16, but they sum products in a
different order (fp32 on the tensor cores, float64 on the CPU), so a stored
element may round to the neighbouring bf16 value on one side: a difference of
one bf16 ulp (at most 2^-7 of its magnitude; bf16 keeps 8 significant bits),
which later layers carry forward.  A worst-case (absolute-value) propagation
of these differences through three 256-wide layers grows by the sum of |W|
per layer and gives bounds far above the gradients themselves, so
``grad_error_bound`` treats them as independent, zero-mean differences and
propagates their variances.  A stored element flips when a rounding boundary
falls between the two sides' unrounded values; with the boundary anywhere in
the ulp, that happens with probability (their difference) / ulp, taken as
min(1, (summation bound + 3 standard deviations of the carried difference) /
ulp), so the element adds that probability times ulp^2 to its variance.
Products carry variances through squared weights and activations, the softmax
passes a logit difference on with its Jacobian, a ReLU whose input is within
three standard deviations of zero may switch on one side only (its whole term
is added), and fp32 summation of n terms differs by at most n 2^-24 of the sum
of |terms| (doubled for the tensor cores' accumulation).  The element-wise
tolerance is 6 standard deviations plus that summation term.
"""
import numpy as np

from oracle import mlp_ref

U_BF16 = 2.0 ** -7   # one bf16 ulp, relative
U_F32 = 2.0 ** -24   # fp32 unit roundoff
SIGMAS = 6.0


def ulp_bf16(x):
    """The spacing of bf16 values at |x| (tiny for zeros)."""
    a = np.maximum(np.abs(np.asarray(x, np.float64)), 2.0 ** -126)
    return 2.0 ** (np.floor(np.log2(a)) - 7)


def bf16_bits(values):
    """uint16 bit patterns of float values rounded to bf16 (ties to even)."""
    r = mlp_ref.bf16(values).astype(np.float32)
    return (r.view(np.uint32) >> 16).astype(np.uint16)


def _stored_var(x, var_in, acc):
    """Variance of a stored bf16 element's difference: what it carries, plus
    one ulp^2 times the chance that its rounding flips."""
    u = ulp_bf16(x)
    p = np.minimum(1.0, (acc + 3.0 * np.sqrt(var_in)) / u)
    return var_in + np.where(x != 0, p * u * u, 0.0)


def grad_error_bound(params, feats, labels, steps):
    """Element-wise tolerance (flat parameter layout) for |GPU - CPU| gradients."""
    q = mlp_ref.bf16
    layers = mlp_ref.unflatten(params)
    Wq = [q(W) for W, _ in layers]
    W2 = [w * w for w in Wq]
    M = len(labels)
    # forward: activations, variances of their differences, summation bounds
    X = [q(feats)]
    V = [np.zeros_like(X[0])]
    pre = [None]  # pre-activations and their variances, per hidden layer
    for l in range(3):
        b = layers[l][1]
        A = X[l] @ Wq[l].T + b
        acc = (X[l].shape[1] + 1) * U_F32 * (np.abs(X[l]) @ np.abs(Wq[l]).T + np.abs(b))
        var_pre = V[l] @ W2[l].T + acc * acc
        unsure = np.abs(A) <= 3.0 * np.sqrt(var_pre)
        H = q(np.maximum(A, 0.0))
        pre.append((A, var_pre))
        X.append(H)
        V.append(_stored_var(H, var_pre, acc) + np.where(unsure, A * A, 0.0))
    b3 = layers[3][1]
    Z = X[3] @ Wq[3].T + b3
    accZ = (X[3].shape[1] + 1) * U_F32 * (np.abs(X[3]) @ np.abs(Wq[3]).T + np.abs(b3))
    VZ = V[3] @ W2[3].T + accZ * accZ
    # cross-entropy gradient: dp_t = p_t (delta_t - sum_s p_s delta_s)
    dZ = mlp_ref.ce_grad(Z, labels, steps, M)
    T = Z.shape[1]
    mask = np.arange(T)[None, :] < np.asarray(steps)[:, None]
    valid = (np.asarray(labels) >= 0)[:, None]
    onehot = np.arange(T)[None, :] == np.asarray(labels)[:, None]
    P = np.where(mask & valid, dZ * M + np.where(onehot, 1.0, 0.0), 0.0)
    vz = np.where(mask, VZ, 0.0)
    var_p = P * P * (vz + (P * P * vz).sum(axis=1, keepdims=True))
    dY = q(dZ)
    accZg = 1e-6 * (P + 1.0) * (mask & valid) / M  # fp32 exp, sum and divide
    VdY = _stored_var(dY, var_p / (M * M) + accZg ** 2, accZg)
    tol = [None] * 4
    for l in range(3, -1, -1):
        Xl, Vl = X[l], V[l]
        K = Xl.shape[0]
        var_W = VdY.T @ (Xl * Xl) + (dY * dY).T @ Vl
        var_b = VdY.sum(axis=0)
        accW = (K + 16) * 2 * U_F32 * (np.abs(dY).T @ np.abs(Xl))
        accb = (K + 16) * 2 * U_F32 * np.abs(dY).sum(axis=0)
        tol[l] = (SIGMAS * np.sqrt(var_W) + accW, SIGMAS * np.sqrt(var_b) + accb)
        if l == 0:
            break
        dX = dY @ Wq[l]
        accX = (Wq[l].shape[0] + 16) * 2 * U_F32 * (np.abs(dY) @ np.abs(Wq[l]))
        var_dX = VdY @ W2[l] + accX * accX
        dYn = q(np.where(Xl > 0, dX, 0.0))
        A, var_pre = pre[l]
        unsure = np.abs(A) <= 3.0 * np.sqrt(var_pre)  # the ReLU may be on at one side only
        VdY = _stored_var(dYn, np.where(Xl > 0, var_dX, 0.0), np.where(Xl > 0, accX, 0.0)) + \
            np.where(unsure, dX * dX, 0.0)
        dY = dYn
    return mlp_ref.flatten(tol)
