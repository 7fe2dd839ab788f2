"""Reference of the small MLP used as a learned coarse-grid correction (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Network (batch rows, FP64): h1 = relu(X W1^T + b1), h2 = relu(h1 W2^T + b2),
Y = h2 W3^T + b3; loss L = mean((Y - T)^2) over all B*n entries.  Gradients
by the chain rule written out step by step (checked against central finite
differences in the tests).
"""
from __future__ import annotations

import numpy as np


def forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    Z1 = X @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3.T + b3
    return Y, (X, Z1, H1, Z2, H2)


def loss(params, X, T):
    Y, _ = forward(params, X)
    return float(np.mean((Y - T) ** 2))


def grads(params, X, T):
    W1, b1, W2, b2, W3, b3 = params
    Y, (X, Z1, H1, Z2, H2) = forward(params, X)
    dY = 2.0 * (Y - T) / Y.size
    dW3 = dY.T @ H2
    db3 = dY.sum(axis=0)
    dH2 = dY @ W3
    dZ2 = dH2 * (Z2 > 0)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dH1 = dZ2 @ W2
    dZ1 = dH1 * (Z1 > 0)
    dW1 = dZ1.T @ X
    db1 = dZ1.sum(axis=0)
    return [dW1, db1, dW2, db2, dW3, db3]


def init(n, hidden, seed=0):
    """He-style initial weights (the GPU side receives these as inputs)."""
    rng = np.random.default_rng(seed)
    W1 = rng.standard_normal((hidden, n)) * np.sqrt(2.0 / n)
    W2 = rng.standard_normal((hidden, hidden)) * np.sqrt(2.0 / hidden)
    W3 = rng.standard_normal((n, hidden)) * np.sqrt(1.0 / hidden)
    return [W1, np.zeros(hidden), W2, np.zeros(hidden), W3, np.zeros(n)]
