"""Pins for the FP64 reference network used to check the CUDA MLP: its
gradient equals central finite differences of its own loss, and the pinball
loss has the textbook values."""
import numpy as np

from oracle import mlp as omlp


def test_pinball_loss_values():
    # u = t - y: tau*u for u >= 0, (tau-1)*u for u < 0
    y = np.array([0.0, 0.0, 2.0])
    t = np.array([1.0, -1.0, 2.0])
    assert abs(omlp.pinball(y, t, 0.9) - (0.9 * 1 + 0.1 * 1 + 0) / 3) < 1e-15


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, hid, B = 5, 7, 40
    npar = hid * n_in + hid + hid * hid + hid + hid + 1
    p = rng.normal(0, 0.5, npar)
    X = rng.normal(0, 1, (B, n_in))
    t = rng.normal(0, 1, B)
    mean, std = X.mean(0), X.std(0)
    g, _ = omlp.grad(p, X, t, 0.9, mean, std, n_in, hid)
    eps = 1e-6
    num = np.zeros_like(p)
    for i in range(npar):
        d = np.zeros_like(p)
        d[i] = eps
        lp = omlp.pinball(omlp.forward(p + d, X, mean, std, n_in, hid)[0], t, 0.9)
        lm = omlp.pinball(omlp.forward(p - d, X, mean, std, n_in, hid)[0], t, 0.9)
        num[i] = (lp - lm) / (2 * eps)
    # the loss is piecewise linear: compare where no residual changes sign
    np.testing.assert_allclose(g, num, rtol=1e-5, atol=1e-7)
