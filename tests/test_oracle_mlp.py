"""Pins for the FP64 cost-model oracle: the analytic gradient against central
finite differences of the forward, hand-set networks with closed-form
outputs, and the BF16 rounding rule."""
import numpy as np

from oracle import mlp


def _rand(seed, n=40):
    rng = np.random.default_rng(seed)
    p = rng.normal(0, 0.3, mlp.NPARAMS)
    X = rng.uniform(0, 1, (n, mlp.IN))
    T = rng.normal(0, 1, n)
    return p, X, T


def test_gradient_matches_finite_differences():
    p, X, T = _rand(1)
    _, g = mlp.loss_grad(p, X, T)
    h = 1e-6
    idx = np.r_[0:40, mlp.B1:mlp.B1 + 10, mlp.W2:mlp.W2 + 60, mlp.B2:mlp.B2 + 10, mlp.W3:mlp.NPARAMS]
    for i in idx:
        e = np.zeros(mlp.NPARAMS)
        e[i] = h
        fd = (mlp.loss(p + e, X, T) - mlp.loss(p - e, X, T)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i
    L, _ = mlp.loss_grad(p, X, T)
    assert abs(L - mlp.loss(p, X, T)) < 1e-12


def test_closed_form_networks():
    X = np.linspace(-2, 2, 9)[:, None] * np.ones((1, mlp.IN))
    p = np.zeros(mlp.NPARAMS)
    p[mlp.B3] = 1.25
    np.testing.assert_allclose(mlp.forward(p, X), 1.25)
    # y = 2 * relu(relu(x0)) + 0.5
    p[mlp.W1 + 0 * mlp.IN + 0] = 1.0
    p[mlp.W2 + 0 * mlp.HID + 0] = 1.0
    p[mlp.W3 + 0] = 2.0
    p[mlp.B3] = 0.5
    np.testing.assert_allclose(mlp.forward(p, X), 2 * np.maximum(X[:, 0], 0) + 0.5)
    # a bias that keeps unit 1 of layer 2 active adds w3[1] * b2[1]
    p[mlp.B2 + 1] = 3.0
    p[mlp.W3 + 1] = -0.25
    np.testing.assert_allclose(mlp.forward(p, X), 2 * np.maximum(X[:, 0], 0) + 0.5 - 0.75)


def test_bf16_rounding():
    one = np.float32(1.0)
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, 1 + 2 ** -7, -3.0, 2 ** -126], dtype=np.float32)
    want = np.array([1.0, 1.0, 1 + 2 ** -7, 1 + 2 ** -7, -3.0, 2 ** -126], dtype=np.float32)
    np.testing.assert_array_equal(mlp.bf16(vals), want)
    assert mlp.bf16(one) == one
