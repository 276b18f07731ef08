"""FP64 reference of the learned initialiser's network (numpy).

TEST INFRASTRUCTURE: only the test suite may use it.  A three-layer perceptron
x -> GELU(W1 x + b1) -> GELU(W2 h1 + b2) -> W3 h2 + b3 with the mean-squared
loss L = sum((y - t)^2) / (B * n_out) or its phase-invariant form (each
target row rotated by the global phase that best matches the output row),
the gradients by the chain rule, and
one Adam step (Kingma & Ba 2015, bias-corrected moments).  GELU is the exact
form x * Phi(x) = x/2 (1 + erf(x / sqrt 2)).

Parameters travel as one flat vector in the order W1 [h1][in], b1, W2 [h2][h1],
b2, W3 [out][h2], b3 (row-major), the layout libtmr uses.
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def shapes(n_in, n_h1, n_h2, n_out):
    return [(n_h1, n_in), (n_h1,), (n_h2, n_h1), (n_h2,), (n_out, n_h2), (n_out,)]


def unflatten(theta, dims):
    out, o = [], 0
    for s in shapes(*dims):
        n = int(np.prod(s))
        out.append(np.asarray(theta[o:o + n], dtype=np.float64).reshape(s))
        o += n
    return out


def flatten(parts):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def forward(theta, dims, X):
    W1, b1, W2, b2, W3, b3 = unflatten(theta, dims)
    Z1 = X @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss_grad(theta, dims, X, T):
    """L = mean squared error over every output; returns (L, flat gradient)."""
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unflatten(theta, dims)
    Y, (X, Z1, H1, Z2, H2) = forward(theta, dims, X)
    B, n_out = Y.shape
    L = np.sum((Y - T) ** 2) / (B * n_out)
    dY = 2.0 * (Y - T) / (B * n_out)
    dW3 = dY.T @ H2
    db3 = dY.sum(0)
    dZ2 = (dY @ W3) * gelu_grad(Z2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(0)
    return L, flatten([dW1, db1, dW2, db2, dW3, db3])


def align_targets(Y, T):
    """Each target row, read as the complex vector t = T[:n] + i T[n:] (n =
    n_out / 2), rotated by the global phase that best aligns it with the
    output row y = Y[:n] + i Y[n:]: t e^{-i a} with e^{i a} = c / |c|,
    c = sum conj(y) t (no rotation where c = 0).  Returned in the same real
    layout.  Rows of T are determined only up to a global phase (a TM row
    is), so the loss compares each output with the nearest rotation of its
    target."""
    Y = np.asarray(Y, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    n = Y.shape[1] // 2
    y = Y[:, :n] + 1j * Y[:, n:]
    t = T[:, :n] + 1j * T[:, n:]
    c = np.sum(np.conj(y) * t, axis=1)
    ac = np.abs(c)
    rot = np.where(ac > 0, np.conj(c) / np.where(ac > 0, ac, 1.0), 1.0)
    tr = t * rot[:, None]
    return np.concatenate([tr.real, tr.imag], axis=1)


def loss_grad_phase(theta, dims, X, T):
    """Phase-invariant loss L = sum_b min_a ||y_b - t_b e^{-i a}||^2 / (B n_out)
    (outputs and targets as complex rows, see align_targets) and its gradient.
    The minimum over a is attained at the aligning rotation, so by the
    envelope theorem dL/dY = 2 (Y - align(T)) / (B n_out): the mean-squared
    loss against the aligned targets, with the rotation held fixed."""
    Y, _ = forward(theta, dims, np.asarray(X, dtype=np.float64))
    return loss_grad(theta, dims, X, align_targets(Y, T))


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step t (1-based); returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** t)
    vh = v / (1 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
