"""CPU oracle of the cost model's network (test infrastructure only).

The network, loss and Adam update written out in float64 numpy, following
their definitions: h1 = tanh(W1 x + b1), h2 = tanh(W2 h1 + b2),
y = w3 . h2 + b3, L = mean (y - t)^2 (the layout of the flat parameter
vector is the library's: W1 [H][D], b1 [H], W2 [H][H], b2 [H], w3 [H], b3).
The gradient is the chain rule written by hand; it is pinned against
central finite differences of the loss (tests/test_mlp_oracle.py), which
share no code with it.  Adam follows Kingma & Ba (ICLR 2015), Algorithm 1.
"""

import numpy as np


def split(p, D, H):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * D].reshape(H, D); o += H * D
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def param_count(D, H):
    return H * D + H + H * H + H + H + 1


def forward(p, X, D, H):
    W1, b1, W2, b2, w3, b3 = split(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ w3 + b3


def loss(p, X, t, D, H):
    y = forward(p, X, D, H)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def grad(p, X, t, D, H):
    """Gradient of the mean squared error by the chain rule."""
    W1, b1, W2, b2, w3, b3 = split(p, D, H)
    X = np.asarray(X, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    n = X.shape[0]
    a1 = X @ W1.T + b1
    h1 = np.tanh(a1)
    a2 = h1 @ W2.T + b2
    h2 = np.tanh(a2)
    y = h2 @ w3 + b3
    dy = 2.0 * (y - t) / n                 # dL/dy
    dw3 = h2.T @ dy
    db3 = dy.sum()
    da2 = np.outer(dy, w3) * (1.0 - h2 ** 2)   # dL/da2
    dW2 = da2.T @ h1
    db2 = da2.sum(axis=0)
    da1 = (da2 @ W2) * (1.0 - h1 ** 2)        # dL/da1
    dW1 = da1.T @ X
    db1 = da1.sum(axis=0)
    return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, [db3]])


def adam(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step; returns (p, m, v) as new arrays (step counts from 1)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mhat = m / (1 - b1 ** step)
    vhat = v / (1 - b2 ** step)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v
