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


def _amb(Z, Zabs, tol):
    """Values whose sign an error of at most tol * Zabs (Zabs the magnitude
    of the terms summed into them) could flip."""
    return np.abs(Z) <= tol * Zabs


def error_bounds(p, X, t, tau, mean, std, n_in, hidden, eps):
    """Per-element error budget of a reduced-precision evaluation of the
    network, its loss gradient and its output, against this module's FP64
    values, written out layer by layer as the FP64 forward and backward
    passes are.  eps is the relative error of each stored operand (inputs,
    weights, hidden activations, back-propagated terms; 2^-8 for bfloat16).

      magnitude: the same passes over absolute values -- |standardised X|,
        |W|, |b|, |dy| -- with every unit counted whose ReLU is active or
        could be flipped; it is the sum of |terms| behind each output and
        gradient element, and a reduced-precision value is within a small
        multiple of eps times it;
      flips: a first-layer pre-activation carries at most 2 eps of its
        magnitude (rounded inputs and weights), a second-layer one 5 eps
        (its rounded inputs and weights, and the first layer's error through
        |W2|), the output 6 eps; a ReLU (or a pinball residual t - y) that
        close to zero may pass or block its whole gradient term, so the terms
        routed through it enter the allowance at full magnitude.

    Returns (y_mag [B], g_mag [P], g_flip [P]) in the flat parameter order."""
    W1, b1, W2, b2, w3, b3 = unpack(p, n_in, hidden)
    y, (Xn, Z1, H1, Z2, H2) = forward(p, X, mean, std, n_in, hidden)
    B = y.size
    aX = np.abs(Xn)
    Z1a = aX @ np.abs(W1).T + np.abs(b1)
    a1 = _amb(Z1, Z1a, 2 * eps)
    on1 = (Z1 > 0) | a1                       # units that may carry a value
    H1a = Z1a * on1
    Z2a = H1a @ np.abs(W2).T + np.abs(b2)
    a2 = _amb(Z2, Z2a, 5 * eps)
    on2 = (Z2 > 0) | a2
    H2a = Z2a * on2
    ya = H2a @ np.abs(w3) + abs(b3[0])
    ay = _amb(np.asarray(t, np.float64) - y, ya, 6 * eps)
    dya = np.full(B, max(tau, 1.0 - tau) / B)
    dyf = np.where(ay, 1.0 / B, 0.0)          # a residual sign flip moves dy by 1/B

    def pack(dW1, db1, dW2, db2, dw3, db3):
        return np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dw3, db3])

    def back(dyv):
        # the backward pass over absolute values, rows weighted by dyv
        dZ2 = np.outer(dyv, np.abs(w3)) * on2
        dH1 = dZ2 @ np.abs(W2)
        dZ1 = dH1 * on1
        return pack(dZ1.T @ aX, dZ1.sum(axis=0), dZ2.T @ H1a, dZ2.sum(axis=0), H2a.T @ dyv,
                    np.array([dyv.sum()])), dH1

    g_mag, dH1a = back(dya)
    # flip allowance: (a) rows whose residual sign may flip, through every
    # carried unit; (b) layer-2 units that may flip: their whole dZ2 term and
    # what it feeds below; (c) layer-1 units that may flip: their whole dZ1
    # term
    fa, _ = back(dyf)
    dZ2f = np.outer(dya, np.abs(w3)) * a2
    dZ1b = (dZ2f @ np.abs(W2)) * on1
    fb = pack(dZ1b.T @ aX, dZ1b.sum(axis=0), dZ2f.T @ H1a, dZ2f.sum(axis=0), np.zeros(hidden),
              np.zeros(1))
    dZ1c = dH1a * a1
    fc = pack(dZ1c.T @ aX, dZ1c.sum(axis=0), np.zeros((hidden, hidden)), np.zeros(hidden),
              np.zeros(hidden), np.zeros(1))
    return ya, g_mag, fa + fb + fc
