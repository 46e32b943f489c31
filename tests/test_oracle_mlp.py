"""Pins of the cost-model network's reference: backpropagation against
central finite differences of the loss, the flat layout, and Adam's first
step (a step of -lr * sign(g) by construction)."""
import numpy as np

from oracle import mlp


def _setup(seed=0, n_in=6, n_hidden=5, n_layers=2, n=9):
    rng = np.random.default_rng(seed)
    shapes = mlp.layer_shapes(n_in, n_hidden, n_layers)
    n_params = sum(fo * fi + fo for fo, fi in shapes)
    params = rng.normal(0, 0.7, n_params)
    X = rng.normal(0, 1, (n, n_in))
    t = rng.normal(0, 1, n)
    mean = rng.normal(0, 0.3, n_in)
    scale = rng.uniform(0.5, 2.0, n_in)
    return params, mean, scale, X, t, (n_in, n_hidden, n_layers)


def test_layout_counts():
    shapes = mlp.layer_shapes(32, 128, 3)
    assert shapes == [(128, 32), (128, 128), (128, 128), (1, 128)]
    assert sum(fo * fi + fo for fo, fi in shapes) == 32 * 128 + 128 + 2 * (128 * 128 + 128) + 128 + 1


def test_backprop_matches_finite_differences():
    params, mean, scale, X, t, dims = _setup()
    g = mlp.gradients(params, mean, scale, X, t, *dims)
    h = 1e-6
    for i in range(len(params)):
        p1, p2 = params.copy(), params.copy()
        p1[i] += h
        p2[i] -= h
        fd = (mlp.loss(p1, mean, scale, X, t, *dims) - mlp.loss(p2, mean, scale, X, t, *dims)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_linear_network_is_least_squares_gradient():
    # no hidden layer: y = w.x + b, dL/dw = 2/n sum (y - t) x
    rng = np.random.default_rng(3)
    X = rng.normal(size=(7, 4))
    t = rng.normal(size=7)
    params = rng.normal(size=5)
    g = mlp.gradients(params, np.zeros(4), np.ones(4), X, t, 4, 1, 0)
    y = X @ params[:4] + params[4]
    assert np.allclose(g[:4], 2 / 7 * ((y - t)[:, None] * X).sum(0))
    assert np.isclose(g[4], 2 / 7 * (y - t).sum())


def test_adam_first_step_is_signed_lr():
    g = np.array([0.3, -2.0, 1e-3])
    p, _, _ = mlp.adam_step(np.zeros(3), g, np.zeros(3), np.zeros(3), 1, 0.01)
    assert np.allclose(p, -0.01 * np.sign(g), rtol=1e-4)
