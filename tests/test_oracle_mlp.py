"""Pin of the NumPy rank-predictor network: backpropagation against central
finite differences of the loss."""

import numpy as np

from oracle import mlp


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    w = rng.standard_normal(mlp.nweights()) * 0.2
    X = rng.standard_normal((17, 9))
    t = rng.standard_normal(17)
    loss, g = mlp.loss_and_grad(w, X, t)
    idx = rng.choice(len(w), 40, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(w)
        e[i] = h
        fd = (mlp.loss_and_grad(w + e, X, t)[0] - mlp.loss_and_grad(w - e, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_layout_size():
    assert mlp.nweights() == 9025
