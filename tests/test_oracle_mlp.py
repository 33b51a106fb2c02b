"""Pins of the FP64 reference network used to check the GPU training kernels."""
import numpy as np

from oracle import exp_mlp as M


def _sample(seed, n=64):
    rng = np.random.default_rng(seed)
    w = rng.normal(0.0, 0.4, M.PARAMS)
    X = rng.normal(0.0, 1.0, (n, M.IN))
    t = rng.normal(0.0, 2.0, n)
    return w, X, t


def test_gradient_matches_central_differences():
    w, X, t = _sample(1)
    loss, g = M.loss_grad(w, X, t)
    rng = np.random.default_rng(2)
    idx = rng.choice(M.PARAMS, 120, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (M.loss_grad(wp, X, t)[0] - M.loss_grad(wm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1.0 + abs(fd)), i


def test_loss_is_the_mean_squared_error_of_the_forward_pass():
    w, X, t = _sample(3)
    loss, _ = M.loss_grad(w, X, t)
    y = M.forward(w, X)
    assert np.isclose(loss, np.mean((y - t) ** 2), rtol=1e-14)
    # a network with all-zero weights but b3 outputs b3 everywhere
    z = np.zeros(M.PARAMS)
    z[-1] = 1.5
    np.testing.assert_array_equal(M.forward(z, X), np.full(X.shape[0], 1.5))
    # the output-bias gradient of that network is 2 mean(b3 - t)
    assert np.isclose(M.loss_grad(z, X, t)[1][-1], 2.0 * np.mean(1.5 - t), rtol=1e-14)
