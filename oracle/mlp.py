"""FP64 oracle for the tile-choice cost model -- test infrastructure only.

The paper autotunes tile size and unroll factor (Section VI-A).  The cost model
here is a small MLP that predicts log execution time from shape and tile
features: x -> Linear(F, H) -> ReLU -> Linear(H, H) -> ReLU -> Linear(H, 1),
trained with mean squared error and Adam (Kingma & Ba, 2015, Algorithm 1).

Flat parameter order (shared by the library's C-ABI; a data layout, not code):
    W1 [H][F], b1 [H], W2 [H][H], b2 [H], w3 [H], b3 [1]
"""
from __future__ import annotations

import numpy as np


def param_count(F: int, H: int = 64) -> int:
    return H * F + H + H * H + H + H + 1


def unpack(theta: np.ndarray, F: int, H: int = 64):
    t = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = t[o:o + H * F].reshape(H, F); o += H * F
    b1 = t[o:o + H]; o += H
    W2 = t[o:o + H * H].reshape(H, H); o += H * H
    b2 = t[o:o + H]; o += H
    w3 = t[o:o + H]; o += H
    b3 = t[o]
    return W1, b1, W2, b2, w3, b3


def pack(W1, b1, W2, b2, w3, b3) -> np.ndarray:
    return np.concatenate([np.ravel(W1), np.ravel(b1), np.ravel(W2), np.ravel(b2),
                           np.ravel(w3), np.atleast_1d(b3)]).astype(np.float64)


def relu(z):
    return np.maximum(z, 0.0)


def forward(theta, X, H: int = 64):
    """Predictions y (n,) and the intermediate values the backward pass needs."""
    X = np.asarray(X, dtype=np.float64)
    F = X.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(theta, F, H)
    z1 = X @ W1.T + b1
    h1 = relu(z1)
    z2 = h1 @ W2.T + b2
    h2 = relu(z2)
    y = h2 @ w3 + b3
    return y, (X, z1, h1, z2, h2)


def mse(y, t) -> float:
    d = np.asarray(y, np.float64) - np.asarray(t, np.float64)
    return float(np.mean(d * d))


def backward(theta, X, t, H: int = 64):
    """Loss and its gradient with respect to the flat parameter vector, by the
    chain rule through the three layers (ReLU derivative taken as 0 at 0)."""
    y, (X, z1, h1, z2, h2) = forward(theta, X, H)
    F = X.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(theta, F, H)
    n = X.shape[0]
    dy = 2.0 * (y - np.asarray(t, np.float64)) / n        # d loss / d y
    gw3 = h2.T @ dy
    gb3 = dy.sum()
    dh2 = np.outer(dy, w3)
    dz2 = dh2 * (z2 > 0)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dh1 = dz2 @ W2
    dz1 = dh1 * (z1 > 0)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    return mse(y, t), pack(gW1, gb1, gW2, gb2, gw3, gb3)


def adam_step(theta, grad, m, v, step: int, lr: float, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (step counts from 1).  Returns new (theta, m, v)."""
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    theta = np.asarray(theta, np.float64) - lr * mhat / (np.sqrt(vhat) + eps)
    return theta, m, v


def numeric_grad(theta, X, t, h: float = 1e-3, H: int = 64, idx=None):
    """Central finite differences of the loss (for pinning ``backward``)."""
    theta = np.array(theta, dtype=np.float64)
    idx = range(theta.size) if idx is None else idx
    out = {}
    for i in idx:
        tp = theta.copy(); tp[i] += h
        tm = theta.copy(); tm[i] -= h
        out[i] = (mse(forward(tp, X, H)[0], t) - mse(forward(tm, X, H)[0], t)) / (2 * h)
    return out
