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


def _adam_run(steps, g_of_t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, step_fn=om.adam_step, p0=None):
    n = len(g_of_t(1))
    p = np.zeros(n) if p0 is None else np.array(p0, float)
    m = np.zeros(n)
    v = np.zeros(n)
    for t in range(1, steps + 1):
        p, m, v = step_fn(p, g_of_t(t), m, v, lr, b1, b2, eps, t)
    return p, m, v


def test_adam_constant_gradient_closed_form():
    """From zero moments with a constant gradient g, m_t = (1 - b1^t) g and
    v_t = (1 - b2^t) g^2, so the bias-corrected moments are exactly g and g^2
    and every step moves params by -lr g / (|g| + eps)."""
    g = np.array([0.5, -2.0, 1e-3, 0.0, 7.25])
    lr, b1, b2, eps, T = 1e-2, 0.9, 0.999, 1e-8, 25
    p, m, v = _adam_run(T, lambda t: g, lr, b1, b2, eps)
    assert np.allclose(m, (1 - b1 ** T) * g, rtol=1e-14, atol=0)
    assert np.allclose(v, (1 - b2 ** T) * g * g, rtol=1e-13, atol=0)
    assert np.allclose(p, -T * lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-300)


def test_adam_zero_betas_is_a_normalised_step():
    """beta1 = beta2 = 0: no memory and no correction, the step is -lr g / (|g| + eps)."""
    rng = np.random.default_rng(3)
    gs = [rng.standard_normal(6) for _ in range(4)]
    p, _, _ = _adam_run(4, lambda t: gs[t - 1], lr=0.1, b1=0.0, b2=0.0, eps=1e-3)
    want = -sum(0.1 * g / (np.abs(g) + 1e-3) for g in gs)
    assert np.allclose(p, want, rtol=1e-14, atol=1e-15)


def test_adam_hand_two_steps():
    """Two steps by hand: g1 = 1, g2 = -1, b1 = 0.5, b2 = 0.75, lr = 1, eps = 0.
    m1 = 0.5, v1 = 0.25, m_hat = 1, v_hat = 1 -> p1 = -1;
    m2 = 0.25 - 0.5 = -0.25, v2 = 0.1875 + 0.25 = 0.4375,
    m_hat = -0.25 / 0.75 = -1/3, v_hat = 0.4375 / 0.4375 = 1 -> p2 = -1 + 1/3."""
    p, m, v = _adam_run(2, lambda t: np.array([1.0 if t == 1 else -1.0]), lr=1.0, b1=0.5, b2=0.75, eps=0.0)
    assert np.isclose(m[0], -0.25) and np.isclose(v[0], 0.4375)
    assert np.isclose(p[0], -1.0 + 1.0 / 3.0, rtol=1e-15)


def test_adam_pins_catch_a_dropped_bias_correction():
    """A planted mistake (no bias correction) fails the closed-form pin."""
    def no_correction(p, g, m, v, lr, b1, b2, eps, t):
        m = b1 * m + (1 - b1) * g
        v = b2 * v + (1 - b2) * g * g
        return p - lr * m / (np.sqrt(v) + eps), m, v
    g = np.array([0.5, -2.0])
    p, _, _ = _adam_run(5, lambda t: g, 1e-2, 0.9, 0.999, 1e-8, step_fn=no_correction)
    assert not np.allclose(p, -5 * 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-6)
