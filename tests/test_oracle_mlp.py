"""Pins of the FP64 surrogate-network oracle: the analytic gradient against central
differences of the loss, and Adam's first step against its closed form."""
import numpy as np

from oracle import mlp as M


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(0)
    dims = M.layer_dims(3, 5, 4, 2)
    n = sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))
    p = rng.normal(0, 0.5, n)
    x = rng.normal(size=(7, 3))
    t = rng.normal(size=(7, 2))
    _, g = M.loss_and_grad(p, dims, x, t)
    eps = 1e-6
    num = np.zeros(n)
    for i in range(n):
        e = np.zeros(n)
        e[i] = eps
        num[i] = (M.loss_and_grad(p + e, dims, x, t)[0] - M.loss_and_grad(p - e, dims, x, t)[0]) / (2 * eps)
    np.testing.assert_allclose(g, num, rtol=1e-6, atol=1e-9)


def test_loss_is_mean_squared_error_of_forward():
    rng = np.random.default_rng(1)
    dims = M.layer_dims(2, 4, 2, 3)
    n = sum(a * b + b for a, b in zip(dims[:-1], dims[1:]))
    p = rng.normal(size=n)
    x, t = rng.normal(size=(5, 2)), rng.normal(size=(5, 3))
    W0, b0 = p[:8].reshape(4, 2), p[8:12]
    W1, b1 = p[12:24].reshape(3, 4), p[24:27]
    y = np.tanh(x @ W0.T + b0) @ W1.T + b1  # written out for this two-layer case
    loss, _ = M.loss_and_grad(p, dims, x, t)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14


def test_adam_first_step_moves_by_lr_times_sign():
    """At t = 1 the bias-corrected ratio m / sqrt(v) equals g / |g| (up to eps)."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    p1, _, _ = M.adam(p, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    np.testing.assert_allclose(p1, p - 0.01 * np.sign(g), rtol=0, atol=1e-7)
