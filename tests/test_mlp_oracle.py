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


def test_forward_hand_worked_example():
    """2 -> 2 -> 2 -> 1 with non-symmetric weights, worked by hand:
    x = (3, 5), mean (1, 2), std (2, 3) -> standardised (1, 1);
    Z1 = W1 x + b1 = (1+2+0.5, 3-4-1) = (3.5, -2) -> H1 = (3.5, 0);
    Z2 = W2 H1 + b2 = (3.5, 7+1) -> H2 = (3.5, 8);
    y = w3 . H2 + b3 = 7 - 4 + 0.25 = 3.25."""
    W1 = [[1.0, 2.0], [3.0, -4.0]]
    b1 = [0.5, -1.0]
    W2 = [[1.0, -1.0], [2.0, 0.5]]
    b2 = [0.0, 1.0]
    w3 = [2.0, -0.5]
    b3 = [0.25]
    p = np.concatenate([np.ravel(W1), b1, np.ravel(W2), b2, w3, b3])
    y, _ = omlp.forward(p, np.array([[3.0, 5.0]]), np.array([1.0, 2.0]),
                        np.array([2.0, 3.0]), 2, 2)
    assert abs(y[0] - 3.25) < 1e-15
