"""Pins for the FP64 network oracle: analytic backward against central finite differences."""
import numpy as np

from oracle.mlp import N_PARAMS, forward, grad, finite_difference_grad, loss, unpack


def _data(seed=0, n=37):
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, 0.3, N_PARAMS)
    X = rng.normal(0, 1, (n, 32))
    T = rng.normal(0, 1, n)
    return theta, X, T


def test_parameter_count():
    assert N_PARAMS == 6337


def test_backward_matches_finite_differences():
    theta, X, T = _data()
    g = grad(theta, X, T)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(2048, 20, replace=False), 2048 + np.arange(5),
                          2112 + rng.choice(4096, 20, replace=False), 6208 + np.arange(5),
                          6272 + np.arange(5), [6336]])
    fd = finite_difference_grad(theta, X, T, idx)
    assert np.max(np.abs(fd - g[idx])) < 1e-7 * max(1.0, np.max(np.abs(g[idx])))


def test_planted_sign_error_is_caught():
    # flipping the tanh derivative's sign in the chain rule breaks the finite-difference pin
    theta, X, T = _data(2)
    p = unpack(theta)
    y, (Xf, h1, h2) = forward(theta, X)
    dy = 2.0 * (y - T) / X.shape[0]
    wrong = (np.outer(dy, p["W3"]) * (1.0 + h2 ** 2)).T @ h1
    fd = finite_difference_grad(theta, X, T, [2112 + 5])
    assert abs(wrong.ravel()[5] - fd[0]) > 1e-6


def test_forward_of_zero_network_is_bias():
    theta = np.zeros(N_PARAMS)
    theta[-1] = 0.25
    y, _ = forward(theta, np.ones((3, 32)))
    assert np.all(y == 0.25) and loss(theta, np.ones((3, 32)), np.full(3, 0.25)) == 0.0
