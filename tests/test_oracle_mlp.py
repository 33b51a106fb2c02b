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


def test_warm_start_network_gradient_matches_central_differences():
    from oracle import mlp as N
    sizes = [7, 12, 9, 4]
    rng = np.random.default_rng(4)
    P = sum(o * i + o for i, o in zip(sizes[:-1], sizes[1:]))
    w = rng.normal(0.0, 0.5, P)
    X = rng.normal(size=(30, sizes[0]))
    T = rng.normal(size=(30, sizes[-1]))
    loss, g = N.loss_grad(sizes, w, X, T)
    assert np.isclose(loss, np.mean((N.forward(sizes, w, X) - T) ** 2), rtol=1e-14)
    h = 1e-6
    for i in rng.choice(P, 80, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (N.loss_grad(sizes, wp, X, T)[0] - N.loss_grad(sizes, wm, X, T)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * (1.0 + abs(fd)), i
    # the exp-root network is the special case 9 -> 32 -> 32 -> 1
    from oracle import exp_mlp as M
    w9 = rng.normal(0.0, 0.3, M.PARAMS)
    X9 = rng.normal(size=(20, 9))
    t9 = rng.normal(size=20)
    l1, g1 = M.loss_grad(w9, X9, t9)
    l2, g2 = N.loss_grad([9, 32, 32, 1], w9, X9, t9[:, None])
    assert np.isclose(l1, l2, rtol=1e-14) and np.allclose(g1, g2, rtol=1e-12, atol=1e-14)
