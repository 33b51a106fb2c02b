"""FP64 reference of the learned starting point's network (TEST INFRASTRUCTURE ONLY).

The network of the exponential-cone initial guess: 9 inputs -> 32 ReLU -> 32 ReLU -> 1,
parameters packed as W1[32][9], b1[32], W2[32][32], b2[32], w3[32], b3.  The loss is the
mean squared error over a batch.  The gradient is written out by the chain rule, layer by
layer, in plain numpy; it is pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np

IN, HIDDEN = 9, 32
PARAMS = HIDDEN * IN + HIDDEN + HIDDEN * HIDDEN + HIDDEN + HIDDEN + 1


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.size == PARAMS
    o = 0
    W1 = w[o:o + HIDDEN * IN].reshape(HIDDEN, IN); o += HIDDEN * IN
    b1 = w[o:o + HIDDEN]; o += HIDDEN
    W2 = w[o:o + HIDDEN * HIDDEN].reshape(HIDDEN, HIDDEN); o += HIDDEN * HIDDEN
    b2 = w[o:o + HIDDEN]; o += HIDDEN
    w3 = w[o:o + HIDDEN]; o += HIDDEN
    b3 = w[o]
    return W1, b1, W2, b2, w3, b3


def forward(w, X):
    """Network output for each row of X (n x 9)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss_grad(w, X, t):
    """Mean squared error of the outputs against t and its gradient (packed like w)."""
    W1, b1, W2, b2, w3, b3 = unpack(w)
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    B = X.shape[0]
    z1 = X @ W1.T + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2.T + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ w3 + b3
    e = y - t
    loss = np.mean(e * e)
    dy = 2.0 * e / B                     # dloss / dy
    g_w3 = h2.T @ dy
    g_b3 = dy.sum()
    d2 = np.outer(dy, w3) * (z2 > 0.0)   # dloss / dz2
    g_W2 = d2.T @ h1
    g_b2 = d2.sum(axis=0)
    d1 = (d2 @ W2) * (z1 > 0.0)          # dloss / dz1
    g_W1 = d1.T @ X
    g_b1 = d1.sum(axis=0)
    grad = np.concatenate([g_W1.ravel(), g_b1, g_W2.ravel(), g_b2, g_w3, [g_b3]])
    return loss, grad
