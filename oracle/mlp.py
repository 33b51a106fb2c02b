"""FP64 reference of the warm-start network (TEST INFRASTRUCTURE ONLY).

A fully connected network with ReLU after every layer but the last; parameters packed
per layer as W_l (out x in, row-major) then b_l; loss = mean squared error over all
outputs of all rows.  The gradient is the chain rule written out layer by layer; it is
pinned by central finite differences in the tests.
"""
from __future__ import annotations

import numpy as np


def unpack(sizes, w):
    w = np.asarray(w, dtype=np.float64)
    out, o = [], 0
    for din, dout in zip(sizes[:-1], sizes[1:]):
        W = w[o:o + dout * din].reshape(dout, din); o += dout * din
        b = w[o:o + dout]; o += dout
        out.append((W, b))
    assert o == w.size
    return out


def forward(sizes, w, X):
    h = np.asarray(X, dtype=np.float64)
    layers = unpack(sizes, w)
    for l, (W, b) in enumerate(layers):
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if l + 1 < len(layers) else z
    return h


def loss_grad(sizes, w, X, T):
    layers = unpack(sizes, w)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    hs, zs = [X], []
    for l, (W, b) in enumerate(layers):
        z = hs[-1] @ W.T + b
        zs.append(z)
        hs.append(np.maximum(z, 0.0) if l + 1 < len(layers) else z)
    e = hs[-1] - T
    loss = np.mean(e * e)
    dz = 2.0 * e / e.size
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads.append((dz.T @ hs[l], dz.sum(axis=0)))
        if l > 0:
            dz = (dz @ W) * (zs[l - 1] > 0.0)
    flat = []
    for gW, gb in reversed(grads):
        flat += [gW.ravel(), gb]
    return loss, np.concatenate(flat)
