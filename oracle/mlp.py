"""FP64 reference of the k'-predicting network (test infrastructure).

Plain numpy: the network n_in -> hidden -> hidden -> 1 with ReLU, inputs
standardised as (x - mean) / std, and the gradient of the mean pinball loss
(quantile tau: tau*u for u = t - y >= 0, (tau-1)*u otherwise) by the chain
rule written out layer by layer.  Parameters use the flat order of the CUDA
library: W1 [hidden x n_in], b1, W2 [hidden x hidden], b2, w3, b3.
"""
from __future__ import annotations

import numpy as np


def unpack(p, n_in, hidden):
    p = np.asarray(p, np.float64)
    o = 0

    def take(cnt, shape):
        nonlocal o
        a = p[o:o + cnt].reshape(shape)
        o += cnt
        return a

    W1 = take(hidden * n_in, (hidden, n_in))
    b1 = take(hidden, (hidden,))
    W2 = take(hidden * hidden, (hidden, hidden))
    b2 = take(hidden, (hidden,))
    w3 = take(hidden, (hidden,))
    b3 = take(1, (1,))
    assert o == p.size
    return W1, b1, W2, b2, w3, b3


def forward(p, X, mean, std, n_in, hidden):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, hidden)
    Xn = (np.asarray(X, np.float64) - mean) / std
    Z1 = Xn @ W1.T + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2.T + b2
    H2 = np.maximum(Z2, 0.0)
    y = H2 @ w3 + b3[0]
    return y, (Xn, Z1, H1, Z2, H2)


def pinball(y, t, tau):
    u = np.asarray(t, np.float64) - y
    return float(np.mean(np.where(u >= 0, tau * u, (tau - 1.0) * u)))


def grad(p, X, t, tau, mean, std, n_in, hidden):
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, hidden)
    y, (Xn, Z1, H1, Z2, H2) = forward(p, X, mean, std, n_in, hidden)
    B = y.size
    u = np.asarray(t, np.float64) - y
    dy = ((u < 0).astype(np.float64) - tau) / B          # d mean-loss / dy
    dw3 = H2.T @ dy
    db3 = np.array([dy.sum()])
    dZ2 = np.outer(dy, w3) * (Z2 > 0)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(axis=0)
    dZ1 = (dZ2 @ W2) * (Z1 > 0)
    dW1 = dZ1.T @ Xn
    db1 = dZ1.sum(axis=0)
    g = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])
    return g, pinball(y, t, tau)
