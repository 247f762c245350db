"""FP64 numpy reference of the cost model's network and of its loss gradient.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py). Three fully connected layers of width
64 with ReLU: h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = w3 . h2 + b3, loss =
mean over samples of (y - t)^2. Parameters are one flat vector in the library's order:
W1 (64 x d, row = output unit), b1 (64), W2 (64 x 64), b2 (64), w3 (64), b3 (1).
"""
from __future__ import annotations

import numpy as np

WIDTH = 64


def n_params(d: int) -> int:
    return WIDTH * d + WIDTH + WIDTH * WIDTH + WIDTH + WIDTH + 1


def unpack(p: np.ndarray, d: int):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + WIDTH * d].reshape(WIDTH, d); o += WIDTH * d
    b1 = p[o:o + WIDTH]; o += WIDTH
    W2 = p[o:o + WIDTH * WIDTH].reshape(WIDTH, WIDTH); o += WIDTH * WIDTH
    b2 = p[o:o + WIDTH]; o += WIDTH
    w3 = p[o:o + WIDTH]; o += WIDTH
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, x):
    W1, b1, W2, b2, w3, b3 = unpack(p, x.shape[1])
    h1 = np.maximum(x @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss(p, x, t) -> float:
    return float(np.mean((forward(p, x) - t) ** 2))


def grad(p, x, t):
    """(loss, dloss/dp) by back-propagation."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    W1, b1, W2, b2, w3, b3 = unpack(p, x.shape[1])
    z1 = x @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    n = x.shape[0]
    dy = 2.0 * (y - t) / n
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    dz2 = np.outer(dy, w3) * (z2 > 0)
    g_W2 = dz2.T @ h1
    g_b2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (z1 > 0)
    g_W1 = dz1.T @ x
    g_b1 = dz1.sum(0)
    g = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return float(np.mean((y - t) ** 2)), g
