"""FP64 oracle of the cost-model network -- TEST INFRASTRUCTURE ONLY.

A 3-layer perceptron y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 with the
mean squared error L = (1/N) sum_n (y_n - t_n)^2, its forward pass and its
gradients by hand-derived backpropagation (chain rule), in numpy FP64.
The parameter vector is packed as W1 (H x F, row-major), b1 (H), W2 (H x H),
b2 (H), W3 (1 x H), b3 (1) -- the same packing the GPU kernels use, which is
a storage convention, not shared code.
"""
from __future__ import annotations

import numpy as np


def param_count(F: int, H: int) -> int:
    return H * F + H + H * H + H + H + 1


def unpack(p, F: int, H: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * F].reshape(H, F); o += H * F
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H].reshape(1, H); o += H
    b3 = p[o:o + 1]; o += 1
    return W1, b1, W2, b2, W3, b3


def forward(p, X, F: int, H: int):
    """y (N,) and the activations, for inputs X (N x F)."""
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H)
    X = np.asarray(X, dtype=np.float64)
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = (h2 @ W3.T + b3)[:, 0]
    return y, (z1, h1, z2, h2)


def loss(p, X, T, F: int, H: int) -> float:
    y, _ = forward(p, X, F, H)
    return float(np.mean((y - np.asarray(T, dtype=np.float64)) ** 2))


def grad(p, X, T, F: int, H: int) -> np.ndarray:
    """dL/dp for the mean squared error, by backpropagation."""
    W1, b1, W2, b2, W3, b3 = unpack(p, F, H)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    N = X.shape[0]
    y, (z1, h1, z2, h2) = forward(p, X, F, H)
    dy = 2.0 * (y - T) / N                      # (N,)
    gW3 = dy @ h2                               # (H,)
    gb3 = np.array([dy.sum()])
    dh2 = np.outer(dy, W3[0]) * (z2 > 0)        # (N, H)
    gW2 = dh2.T @ h1                            # (H, H)
    gb2 = dh2.sum(axis=0)
    dh1 = (dh2 @ W2) * (z1 > 0)                 # (N, H)
    gW1 = dh1.T @ X                             # (H, F)
    gb1 = dh1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])


def numeric_grad(p, X, T, F: int, H: int, idx, h: float = 1e-6) -> np.ndarray:
    """Central finite differences of the loss for the parameters in idx."""
    p = np.array(p, dtype=np.float64)
    out = []
    for i in idx:
        a = p.copy(); a[i] += h
        b = p.copy(); b[i] -= h
        out.append((loss(a, X, T, F, H) - loss(b, X, T, F, H)) / (2 * h))
    return np.array(out)


def adam_step(p, g, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015) with bias correction."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v
