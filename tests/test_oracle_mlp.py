"""Pins of the predictor's CPU oracle (oracle/mlp.py): central finite
differences for the gradient, a network whose output has a closed form, and
the closed form of Adam's first step."""
import numpy as np

from oracle import mlp


def rand_params(seed, scale=0.3):
    return np.random.default_rng(seed).normal(0.0, scale, mlp.N_PARAMS)


def test_param_count_matches_library_layout():
    assert mlp.N_PARAMS == 64 * 16 + 64 + 64 * 64 + 64 + 3 * 64 + 3 == 5443


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = rand_params(2)
    x = rng.normal(size=(7, 16))
    t = rng.normal(size=(7, 3))
    w = np.array([1.0, 0.5, 2.0])
    g = mlp.backward(p, x, t, w)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, size=60, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = h
        fd = (mlp.loss(p + e, x, t, w) - mlp.loss(p - e, x, t, w)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_closed_form_network():
    # W1 copies the 16 inputs into the first 16 hidden units, W2 sums them in
    # unit 0, W3 reads unit 0 into output 1 and b3 = (1, 0, -2): for
    # non-negative inputs y = (1, sum(x), -2).
    d = {name: np.zeros(shape) for name, shape in mlp.SHAPES}
    d["W1"][:16, :16] = np.eye(16)
    d["W2"][0, :16] = 1.0
    d["W3"][1, 0] = 1.0
    d["b3"][:] = [1.0, 0.0, -2.0]
    x = np.abs(np.random.default_rng(3).normal(size=(5, 16)))
    y, _ = mlp.forward(mlp.pack(d), x)
    np.testing.assert_allclose(y, np.stack([np.ones(5), x.sum(1), -2 * np.ones(5)], 1), rtol=1e-14)
    # negative inputs are cut by the ReLU
    y, _ = mlp.forward(mlp.pack(d), -x)
    np.testing.assert_allclose(y[:, 1], 0.0)


def test_adam_first_step_closed_form():
    # from m = v = 0: mhat = g, vhat = g^2, step = lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    p0 = np.zeros(4)
    p1, m, v = mlp.adam_step(p0, g, np.zeros(4), np.zeros(4), lr=0.1, step=1)
    np.testing.assert_allclose(p1, -0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)
    np.testing.assert_allclose(m, 0.1 * g)
    np.testing.assert_allclose(v, 0.001 * g * g)
