"""FP64 CPU reference of the learned warm start: TEST INFRASTRUCTURE ONLY.

Only the test suite, the smoke check and the benchmark's CPU leg use this
module; the product path never imports it.  It shares no code with the CUDA
library.

The network is this project's design for the learned warm start of the push
solver (the paper has no learned part; a push from any start converges to the
same certificate, Lemma 3 and Lemma 5).  With a_vj the CSR weights (row v lists
the nodes v listens to), d_v = sum_j a_vj and din_v the number of nodes that
listen to v:

    features   x_v = [s_v, log(1 + d_v), log(1 + din_v), m_v],
               m_v = sum_j a_vj s_j / d_v            (0 when d_v = 0)
    layer l    h^l_v = relu(W^l_s^T h^{l-1}_v + W^l_n^T g^{l-1}_v + b^l),
               g^{l-1}_v = sum_j a_vj h^{l-1}_j / d_v (0 when d_v = 0),
               h^0 = x, l = 1, 2, 3, width 64
    output     z0_v = b_v + w_o . h^3_v + b_o,
               b_v = (s_v + d_v m_v) / (1 + d_v)   (one Jacobi step from s)
    loss       L = (1/n) sum_v (z0_v - z_v)^2

The base term b_v is the equilibrium equation of node v (Section 3.2) with its
neighbours' values taken as their opinions; the network learns the correction.

Parameters are one flat FP32 vector, in this order: for l = 1, 2, 3 the
matrices W^l_s [F_in][64] and W^l_n [F_in][64] (row-major) and b^l [64], then
w_o [64] and b_o [1]; F_in = 4 for l = 1, else 64.

``bf16=True`` rounds to bfloat16 at the points where the GPU kernels keep
bfloat16 values: the stored activations h^l (and x), the aggregated g^l, the
weight matrices and the pre-activation gradients fed to the GEMMs.  Everything
else is FP64.
"""
from __future__ import annotations

import numpy as np

HIDDEN = 64
LAYERS = 3
F_IN = 4


def layer_dims():
    return [(F_IN if l == 0 else HIDDEN, HIDDEN) for l in range(LAYERS)]


def param_count() -> int:
    return sum(2 * fi * fo + fo for fi, fo in layer_dims()) + HIDDEN + 1


def unpack(theta):
    """Flat parameter vector -> list of (Ws, Wn, b) per layer, w_o, b_o (FP64 views)."""
    theta = np.asarray(theta, np.float64)
    assert theta.shape == (param_count(),)
    out, at = [], 0
    for fi, fo in layer_dims():
        ws = theta[at:at + fi * fo].reshape(fi, fo); at += fi * fo
        wn = theta[at:at + fi * fo].reshape(fi, fo); at += fi * fo
        b = theta[at:at + fo]; at += fo
        out.append((ws, wn, b))
    wo = theta[at:at + HIDDEN]; at += HIDDEN
    bo = theta[at]
    return out, wo, bo


def pack(layers, wo, bo) -> np.ndarray:
    parts = []
    for ws, wn, b in layers:
        parts += [np.ravel(ws), np.ravel(wn), np.ravel(b)]
    parts += [np.ravel(wo), np.array([bo], np.float64)]
    return np.concatenate(parts).astype(np.float64)


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), through FP32 as the GPU does."""
    f = np.asarray(x, np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _mean_op(n, row_ptr, col, w):
    """g = D^{-1} A h as a function, plus its adjoint (the transpose, for backward)."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    a = np.ones(col.shape[0]) if w is None else np.asarray(w, np.float64)
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    d = np.bincount(rows, weights=a, minlength=n)
    scale = np.where(d > 0, 1.0 / np.where(d > 0, d, 1.0), 0.0)
    coef = a * scale[rows]  # a_vj / d_v per nonzero

    def fwd(h):
        out = np.zeros((n, h.shape[1]))
        np.add.at(out, rows, coef[:, None] * h[col])
        return out

    def adj(gbar):
        out = np.zeros((n, gbar.shape[1]))
        np.add.at(out, col, coef[:, None] * gbar[rows])
        return out

    return fwd, adj, d


def features(n, row_ptr, col, w, s):
    """x_v = [s_v, log(1 + d_v), log(1 + din_v), m_v] (FP64)."""
    fwd, _, d = _mean_op(n, row_ptr, col, w)
    din = np.bincount(np.asarray(col, np.int64), minlength=n).astype(np.float64)
    s = np.asarray(s, np.float64)
    m = fwd(s[:, None])[:, 0]
    return np.stack([s, np.log1p(d), np.log1p(din), m], axis=1)


def base_term(n, row_ptr, col, w, s):
    """b_v = (s_v + d_v m_v) / (1 + d_v): one Jacobi step of (I + L) z = s from z = s."""
    fwd, _, d = _mean_op(n, row_ptr, col, w)
    s = np.asarray(s, np.float64)
    m = fwd(s[:, None])[:, 0]
    return (s + d * m) / (1.0 + d)


def forward(theta, n, row_ptr, col, w, s, bf16=False):
    """z0 and the saved activations (a dict) of the network."""
    layers, wo, bo = unpack(theta)
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    fwd, adj, _ = _mean_op(n, row_ptr, col, w)
    h = rnd(features(n, row_ptr, col, w, s))
    saved = {"H": [h], "G": [], "pre": []}
    for ws, wn, b in layers:
        g = rnd(fwd(h))
        pre = h @ rnd(ws) + g @ rnd(wn) + b
        h = rnd(np.maximum(pre, 0.0))
        saved["G"].append(g)
        saved["pre"].append(pre)
        saved["H"].append(h)
    z0 = base_term(n, row_ptr, col, w, s) + h @ wo + bo
    saved["adj"] = adj
    return z0, saved


def loss_and_grad(theta, n, row_ptr, col, w, s, z, bf16=False):
    """Mean squared error of z0 against z and its gradient (manual backward, FP64)."""
    layers, wo, bo = unpack(theta)
    rnd = bf16_round if bf16 else (lambda v: np.asarray(v, np.float64))
    z0, sv = forward(theta, n, row_ptr, col, w, s, bf16)
    adj = sv["adj"]
    diff = z0 - np.asarray(z, np.float64)
    loss = float(np.mean(diff * diff))
    dz = 2.0 * diff / n
    h3 = sv["H"][-1]
    g_wo = h3.T @ dz
    g_bo = float(np.sum(dz))
    dh = np.outer(dz, wo)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        ws, wn, b = layers[l]
        hin, gin, pre = sv["H"][l], sv["G"][l], sv["pre"][l]
        dpre = dh * (pre > 0)
        dq = rnd(dpre)
        grads[l] = (hin.T @ dq, gin.T @ dq, np.sum(dpre, axis=0))
        if l > 0:
            dh = dq @ rnd(ws).T + adj(dq @ rnd(wn).T)
    return loss, pack(grads, g_wo, g_bo)


def adam_step(theta, m, v, grad, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), bias-corrected; returns new (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed: int) -> np.ndarray:
    """Deterministic start: uniform(-1/sqrt(F), 1/sqrt(F)) per weight matrix, zero biases."""
    rng = np.random.default_rng(seed)
    layers = []
    for fi, fo in layer_dims():
        lim = 1.0 / np.sqrt(2 * fi)
        layers.append((rng.uniform(-lim, lim, (fi, fo)), rng.uniform(-lim, lim, (fi, fo)), np.zeros(fo)))
    wo = rng.uniform(-1 / 8, 1 / 8, HIDDEN)
    return pack(layers, wo, 0.0).astype(np.float32).astype(np.float64)
