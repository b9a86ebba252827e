"""Pins of the MLP's CPU reference: its analytic gradient against central
finite differences of its own loss (a check independent of the chain-rule
code), and the loss definition on a hand-computed case."""
import numpy as np

from oracle import mlp as om


def _rand(shape, rng):
    n_in, n_h, n_out = shape
    n = n_h * n_in + n_h + n_h * n_h + n_h + n_out * n_h + n_out
    return rng.standard_normal(n) * 0.5


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    shape = (5, 7, 3)
    p = _rand(shape, rng)
    X = rng.standard_normal((11, 5))
    T = rng.standard_normal((11, 3))
    M = (rng.random((11, 3)) > 0.2).astype(float)
    L, g = om.loss_grad(p, X, T, M, shape)
    assert np.isclose(L, om.loss(p, X, T, M, shape))
    h = 1e-6
    fd = np.empty_like(p)
    for k in range(p.size):
        e = np.zeros_like(p)
        e[k] = h
        fd[k] = (om.loss(p + e, X, T, M, shape) - om.loss(p - e, X, T, M, shape)) / (2 * h)
    assert np.max(np.abs(fd - g)) <= 1e-6 * max(1.0, np.abs(g).max())


def test_loss_on_hand_case():
    shape = (1, 1, 1)
    # W1 = 2, b1 = -1, W2 = 3, b2 = 0, W3 = 0.5, b3 = 1
    p = np.array([2.0, -1.0, 3.0, 0.0, 0.5, 1.0])
    X = np.array([[1.0], [0.25]])          # h1 = relu(1) = 1, relu(-0.5) = 0
    y, _ = om.forward(p, X, shape)         # h2 = 3, 0 -> y = 2.5, 1.0
    assert np.allclose(y[:, 0], [2.5, 1.0])
    T = np.array([[2.0], [0.0]])
    M = np.array([[1.0], [1.0]])
    assert np.isclose(om.loss(p, X, T, M, shape), (0.25 + 1.0) / 2)
