"""Oracle: the rank-predictor network in plain NumPy (FP64).

TEST INFRASTRUCTURE ONLY (see oracle/tree.py).

A multilayer perceptron 9 -> 64 -> 64 -> 64 -> 1 with ReLU hidden layers and a
linear output, loss L = mean_i (y_i - t_i)^2 / 2, gradients by backpropagation
written out layer by layer.  Weight layout (flat, row-major W[in][out]):
W1 b1 W2 b2 W3 b3 W4 b4.
"""

from __future__ import annotations

import numpy as np

DIMS = (9, 64, 64, 64, 1)


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    out, o = [], 0
    for a, b in zip(DIMS[:-1], DIMS[1:]):
        W = w[o:o + a * b].reshape(a, b)
        o += a * b
        bias = w[o:o + b]
        o += b
        out.append((W, bias))
    assert o == len(w)
    return out


def nweights():
    return sum(a * b + b for a, b in zip(DIMS[:-1], DIMS[1:]))


def forward(w, X):
    h = np.asarray(X, dtype=np.float64)
    layers = unpack(w)
    acts = [h]
    for l, (W, b) in enumerate(layers):
        z = h @ W + b
        h = np.maximum(z, 0.0) if l < len(layers) - 1 else z
        acts.append(h)
    return acts[-1][:, 0], acts


def loss_and_grad(w, X, t):
    y, acts = forward(w, X)
    n = len(y)
    d = (y - np.asarray(t, dtype=np.float64))
    loss = 0.5 * np.mean(d * d)
    g = (d / n)[:, None]
    layers = unpack(w)
    grads = []
    for l in range(len(layers) - 1, -1, -1):
        W, _ = layers[l]
        grads.append((acts[l].T @ g, g.sum(axis=0)))
        if l > 0:
            g = (g @ W.T) * (acts[l] > 0)
    flat = []
    for (gW, gb) in reversed(grads):
        flat.append(gW.ravel())
        flat.append(gb)
    return loss, np.concatenate(flat)
