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


def _rand_net(seed, n_in=6, hid=9, B=50):
    rng = np.random.default_rng(seed)
    npar = hid * n_in + hid + hid * hid + hid + hid + 1
    p = rng.normal(0, 0.5, npar)
    X = rng.normal(1, 2, (B, n_in))
    t = rng.normal(0, 1, B)
    return p, X, t, X.mean(0), X.std(0), n_in, hid


def test_error_bounds_dominate_the_values():
    """The magnitude of every output and gradient element (the sum of the
    absolute values of its terms) is at least its absolute value."""
    for seed in range(5):
        p, X, t, mean, std, n_in, hid = _rand_net(seed)
        ya, gm, gf = omlp.error_bounds(p, X, t, 0.9, mean, std, n_in, hid, 2.0 ** -8)
        y, _ = omlp.forward(p, X, mean, std, n_in, hid)
        g, _ = omlp.grad(p, X, t, 0.9, mean, std, n_in, hid)
        assert np.all(ya >= np.abs(y) * (1 - 1e-12))
        assert np.all(gm >= np.abs(g) * (1 - 1e-12) - 1e-15)
        assert np.all(gf >= 0)


def test_error_bounds_equal_the_values_without_cancellation():
    """All weights, inputs and biases non-negative and every residual of the
    same sign: no term cancels, so the magnitudes are the values themselves,
    and with no pre-activation near zero there is no flip allowance."""
    p, X, t, _, _, n_in, hid = _rand_net(7)
    p, X = np.abs(p) + 0.01, np.abs(X) + 0.01
    t = np.full(X.shape[0], 1e6)                  # t > y on every row
    zero, one = np.zeros(n_in), np.ones(n_in)
    ya, gm, gf = omlp.error_bounds(p, X, t, 0.9, zero, one, n_in, hid, 1e-4)
    y, _ = omlp.forward(p, X, zero, one, n_in, hid)
    g, _ = omlp.grad(p, X, t, 0.9, zero, one, n_in, hid)
    np.testing.assert_allclose(ya, y, rtol=1e-12)
    np.testing.assert_allclose(gm, np.abs(g), rtol=1e-12, atol=1e-18)
    assert gf.max() == 0.0


def _perturbed(p, X, t, tau, mean, std, n_in, hid, eps, rng, mode="random"):
    """The network, its output and gradient evaluated with every stored
    operand (inputs, weights, hidden activations, back-propagated terms)
    perturbed by a relative error of at most eps (random, or all +eps, or
    all -eps), as a reduced precision evaluation would."""
    def r(a):
        if mode == "up":
            return a * (1 + eps)
        if mode == "down":
            return a * (1 - eps)
        return a * (1 + rng.uniform(-eps, eps, np.shape(a)))
    W1, b1, W2, b2, w3, b3 = omlp.unpack(p, n_in, hid)
    Xn = r((np.asarray(X, np.float64) - mean) / std)
    Z1 = Xn @ r(W1).T + b1
    H1 = r(np.maximum(Z1, 0))
    Z2 = H1 @ r(W2).T + b2
    H2 = np.maximum(Z2, 0)
    y = H2 @ w3 + b3[0]
    B = y.size
    dy = (((t - y) < 0).astype(np.float64) - tau) / B
    dZ2 = r(np.outer(dy, w3) * (Z2 > 0))
    dZ1 = r((dZ2 @ r(W2)) * (Z1 > 0))
    g = np.concatenate([(dZ1.T @ Xn).ravel(), dZ1.sum(0), (dZ2.T @ H1).ravel(), dZ2.sum(0),
                        H2.T @ dy, [dy.sum()]])
    return y, g


def test_error_bounds_hold_for_perturbed_evaluations():
    """What the bounds are for: an evaluation with relative errors of at most
    eps in each stored operand stays within 6 eps times the magnitude plus
    the flip allowance, element by element -- including evaluations whose
    errors all push the same way (every perturbation at +eps or -eps)."""
    eps = 2.0 ** -8
    for seed in range(30):
        p, X, t, mean, std, n_in, hid = _rand_net(100 + seed)
        rng = np.random.default_rng(seed)
        y64, _ = omlp.forward(p, X, mean, std, n_in, hid)
        g64, _ = omlp.grad(p, X, t, 0.9, mean, std, n_in, hid)
        ya, gm, gf = omlp.error_bounds(p, X, t, 0.9, mean, std, n_in, hid, eps)
        for mode in ("random", "up", "down"):
            y, g = _perturbed(p, X, t, 0.9, mean, std, n_in, hid, eps, rng, mode)
            assert np.all(np.abs(y - y64) <= 6 * eps * ya)
            assert np.all(np.abs(g - g64) <= 6 * eps * gm + gf + 1e-15)
