"""FP64 oracle of the learned surrogate (test infrastructure: only tests/, __graft_entry__.smoke()
and bench.py's CPU baseline may import it).

The paper has no surrogate; this is the plain definition of the network the library trains:
inputs x (8 active-region parameters scaled to [-1, 1]) -> 4 hidden layers of 256 GELU units
-> 129 linear outputs (128 standardised PCA coefficients of the residual spectrum F - F_q, and
the log10 of the predicted RV error in cm/s).  Written with numpy in float64; where the GPU
rounds a GEMM operand to bfloat16 the oracle rounds the same quantity the same way
(`quantize=True`), otherwise everything is exact arithmetic in float64.

  z_l = q(a_{l-1}) q(W_l)^T + b_l,  a_l = GELU(z_l)  (l = 1..4),  y = q(a_4) q(W_5)^T + b_5
  L = sum_b sum_j w_j (y_bj - t_bj)^2 / B
backward (chain rule; q() marks the bfloat16 operands of each product):
  g_5 = q(dL/dy),  dW_5 = g_5^T q(a_4),  db_5 = sum_b g_5
  dz_l = (g_{l+1} q(W_{l+1})) * GELU'(z_l),  g_l = q(dz_l),  dW_l = g_l^T q(a_{l-1}),  db_l = sum_b g_l
GELU(z) = z Phi(z) with the normal CDF Phi (erf form); GELU'(z) = Phi(z) + z phi(z).
Adam (Kingma & Ba 2015, Algorithm 1) with bias correction.
PCA: the top-k right singular vectors of the mean-centred data (numpy SVD).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

N_IN, HIDDEN, N_HIDDEN, N_COEF = 8, 256, 4, 128
N_OUT = N_COEF + 1


def bf16(x) -> np.ndarray:
    """Round to bfloat16 (nearest, ties to even) through float32, returned as float64."""
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / np.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / np.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / np.sqrt(2.0 * np.pi)


def layer_shapes(n_in=N_IN, hidden=HIDDEN, n_hidden=N_HIDDEN, n_out=N_OUT):
    dims = [n_in] + [hidden] * n_hidden + [n_out]
    return [(dims[l + 1], dims[l]) for l in range(len(dims) - 1)]      # (out, in) per layer


def unflatten(flat, shapes):
    """Flat parameter vector [W1 | b1 | W2 | b2 | ...] -> list of (W [out][in], b [out])."""
    out, o = [], 0
    for (n_o, n_i) in shapes:
        W = np.asarray(flat[o:o + n_o * n_i], np.float64).reshape(n_o, n_i)
        o += n_o * n_i
        b = np.asarray(flat[o:o + n_o], np.float64)
        o += n_o
        out.append((W, b))
    return out


def flatten(layers):
    return np.concatenate([np.concatenate([W.ravel(), b]) for W, b in layers])


def forward(layers, X, quantize=True):
    q = bf16 if quantize else (lambda v: np.asarray(v, np.float64))
    a = np.asarray(X, np.float64)
    zs, acts = [], [a]
    for l, (W, b) in enumerate(layers):
        z = q(a) @ q(W).T + b
        zs.append(z)
        if l < len(layers) - 1:
            a = gelu(z)
            acts.append(a)
    return zs[-1], (zs, acts)


def loss_and_grad(layers, X, T, w_out, quantize=True):
    """Loss and gradients (same structure as `layers`) for one batch."""
    q = bf16 if quantize else (lambda v: np.asarray(v, np.float64))
    y, (zs, acts) = forward(layers, X, quantize)
    B = X.shape[0]
    r = y - T
    loss = float(np.sum(w_out * r * r) / B)
    g = q(2.0 * w_out * r / B)
    grads = [None] * len(layers)
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads[l] = (g.T @ q(acts[l]), g.sum(axis=0))
        if l > 0:
            dz = (g @ q(W)) * gelu_grad(zs[l - 1])
            g = q(dz)
    return loss, grads


def adam(flat, grad, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8, mask=None):
    """One Adam step (t = 1, 2, ...); entries where mask is False are left unchanged."""
    m2 = b1 * m + (1 - b1) * grad
    v2 = b2 * v + (1 - b2) * grad * grad
    mh = m2 / (1 - b1 ** t)
    vh = v2 / (1 - b2 ** t)
    new = flat - lr * mh / (np.sqrt(vh) + eps)
    if mask is not None:
        new = np.where(mask, new, flat)
        m2 = np.where(mask, m2, m)
        v2 = np.where(mask, v2, v)
    return new, m2, v2


def pca(X, k):
    """(mean, basis [k][p] with orthonormal rows, singular values [k]) of the rows of X."""
    X = np.asarray(X, np.float64)
    mu = X.mean(axis=0)
    _, s, Vt = np.linalg.svd(X - mu, full_matrices=False)
    return mu, Vt[:k], s[:k]
