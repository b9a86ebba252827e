"""FP64 CPU reference of the variant-predicting MLP -- TEST INFRASTRUCTURE.

Same network and loss as include/sc_mlp.h, written from the definitions:
  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3,
  L = sum mask (y - t)^2 / sum mask,
with the gradients by the chain rule, and the Adam optimiser step
(``adam_step``).  Pinned in the tests by central finite differences of
``loss`` (independent of the backward formulas) and, for Adam, by closed
forms of the moment recursions (constant gradient, beta = 0).
Only the tests may import it.
"""
from __future__ import annotations

import numpy as np


def unpack(params: np.ndarray, n_in: int, n_hidden: int, n_out: int):
    p = np.asarray(params, dtype=np.float64)
    o = 0
    out = []
    for shape in [(n_hidden, n_in), (n_hidden,), (n_hidden, n_hidden), (n_hidden,), (n_out, n_hidden), (n_out,)]:
        k = int(np.prod(shape))
        out.append(p[o:o + k].reshape(shape))
        o += k
    assert o == p.size
    return out


def forward(params, X, shape):
    W1, b1, W2, b2, W3, b3 = unpack(params, *shape)
    X = np.asarray(X, np.float64)
    h1 = np.maximum(X @ W1.T + b1, 0.0)
    h2 = np.maximum(h1 @ W2.T + b2, 0.0)
    return h2 @ W3.T + b3, (X, h1, h2)


def loss(params, X, T, mask, shape) -> float:
    y, _ = forward(params, X, shape)
    d = (y - T) * mask
    return float((d * d).sum() / mask.sum())


def loss_grad(params, X, T, mask, shape):
    W1, b1, W2, b2, W3, b3 = unpack(params, *shape)
    y, (X, h1, h2) = forward(params, X, shape)
    cnt = mask.sum()
    d = (y - T) * mask
    L = float((d * d).sum() / cnt)
    dy = 2.0 * d / cnt
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dh2 = (dy @ W3) * (h2 > 0)
    gW2 = dh2.T @ h1
    gb2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    gW1 = dh1.T @ X
    gb1 = dh1.sum(0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def adam_step(params, grads, m, v, lr: float, beta1: float, beta2: float, eps: float, step: int):
    """One Adam step (Kingma and Ba, "Adam: A method for stochastic
    optimization", ICLR 2015, Algorithm 1), FP64, returning new arrays:

      m <- beta1 m + (1 - beta1) g              (first moment)
      v <- beta2 v + (1 - beta2) g^2            (second raw moment)
      m_hat = m / (1 - beta1^t),  v_hat = v / (1 - beta2^t)   (bias correction, t = step >= 1)
      params <- params - lr m_hat / (sqrt(v_hat) + eps)

    Pinned by closed forms in the tests: with a constant gradient from zero
    moments the corrected moments are exactly g and g^2 at every step."""
    if step < 1:
        raise ValueError("step counts from 1")
    g = np.asarray(grads, np.float64)
    m_new = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v_new = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m_new / (1.0 - beta1 ** step)
    v_hat = v_new / (1.0 - beta2 ** step)
    p_new = np.asarray(params, np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return p_new, m_new, v_new
