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


# ---- BF16 inference forward: hand-set networks -------------------------------
# Every weight below is exactly representable in BF16 (8 significant bits)
# unless stated, so the only differences between forward() and forward_bf16()
# are the roundings the inference path makes: of the input, of each hidden
# activation, of the weights - and none of the output.

def _chain(w1=1.0, b1=0.0, w2=1.0, b2=0.0, w3=1.0, b3=0.0):
    """y = w3 * relu(w2 * relu(w1 * x0 + b1) + b2) + b3 through unit 0."""
    p = np.zeros(mlp.NPARAMS)
    p[mlp.W1] = w1
    p[mlp.B1] = b1
    p[mlp.W2] = w2
    p[mlp.B2] = b2
    p[mlp.W3] = w3
    p[mlp.B3] = b3
    return p


def _x(x0):
    X = np.zeros((1, mlp.IN))
    X[0, 0] = x0
    return X


def test_bf16_forward_rounds_the_first_hidden_layer():
    # a1 = (1 + 2^-7) * 1 + 2^-9 lies 2^-9 above the BF16 value 1 + 2^-7 and
    # 2^-9 - 2^-7 below the next one (spacing 2^-7 in [1, 2)): it rounds down.
    p = _chain(w1=1 + 2 ** -7, b1=2 ** -9)
    assert mlp.forward(p, _x(1.0))[0] == 1 + 2 ** -7 + 2 ** -9
    assert mlp.forward_bf16(p, _x(1.0))[0] == 1 + 2 ** -7
    # with b2 = 3 * 2^-10 the second layer keeps the difference visible:
    # from the rounded h1, a2 = 1 + 11 * 2^-10 rounds down to 1 + 2^-7; from
    # an unrounded h1 it would be 1 + 13 * 2^-10, which rounds up to 1 + 2^-6
    p = _chain(w1=1 + 2 ** -7, b1=2 ** -9, b2=3 * 2 ** -10)
    assert mlp.forward(p, _x(1.0))[0] == 1 + 13 * 2 ** -10
    assert mlp.forward_bf16(p, _x(1.0))[0] == 1 + 2 ** -7


def test_bf16_forward_rounds_the_second_hidden_layer():
    p = _chain(w2=1 + 2 ** -7, b2=2 ** -9)
    assert mlp.forward(p, _x(1.0))[0] == 1 + 2 ** -7 + 2 ** -9
    assert mlp.forward_bf16(p, _x(1.0))[0] == 1 + 2 ** -7


def test_bf16_forward_rounds_inputs_and_weights_but_not_the_output():
    # x0 = 1 + 2^-8 + 2^-10 is 5 * 2^-10 above 1: past the half-way point
    # 2^-8, so BF16 makes it 1 + 2^-7 (3 * 2^-10 more)
    p = _chain()
    x0 = 1 + 2 ** -8 + 2 ** -10
    assert mlp.forward(p, _x(x0))[0] == x0
    assert mlp.forward_bf16(p, _x(x0))[0] == 1 + 2 ** -7
    # with b1 = -2^-9 the rounding of the input decides the hidden unit's
    # cell: rounded, a1 = 1 + 6 * 2^-10 rounds up to 1 + 2^-7; unrounded,
    # a1 = 1 + 3 * 2^-10 would round down to 1
    p = _chain(b1=-2 ** -9)
    assert mlp.forward(p, _x(x0))[0] == 1 + 3 * 2 ** -10
    assert mlp.forward_bf16(p, _x(x0))[0] == 1 + 2 ** -7
    # the same value as a weight of the last layer rounds the same way
    p = _chain(w3=x0)
    assert mlp.forward_bf16(p, _x(1.0))[0] == 1 + 2 ** -7
    # b3 = 2^-12 is a BF16 value; the output 1 + 2^-7 + 2^-12 is not, and
    # stays unrounded
    p = _chain(w1=1 + 2 ** -7, b1=2 ** -9, b3=2 ** -12)
    assert mlp.forward_bf16(p, _x(1.0))[0] == 1 + 2 ** -7 + 2 ** -12


# ---- Adam (Kingma & Ba, Algorithm 1) -----------------------------------------

def test_adam_first_step_is_the_sign_of_the_gradient():
    # t = 1 from zero moments: m_hat = g and v_hat = g^2 exactly (the bias
    # correction divides out the factors 1 - beta), so the step is
    # lr * g / (|g| + eps)
    rng = np.random.default_rng(5)
    p0, g = rng.normal(0, 1, 64), rng.normal(0, 1, 64)
    z = np.zeros(64)
    p1, m1, v1 = mlp.adam_step(p0, g, z, z, 1, 0.01)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-13)
    np.testing.assert_allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)


def test_adam_constant_gradient_moves_by_the_same_step():
    # with g_i = g for every step, m_t = g (1 - b1^t) and v_t = g^2 (1 - b2^t):
    # after bias correction every step is lr * g / (|g| + eps)
    g = np.array([0.5, -2.0, 1e-3, 7.0])
    p = np.zeros(4)
    m = v = np.zeros(4)
    for t in range(1, 51):
        p, m, v = mlp.adam_step(p, g, m, v, t, 1e-3)
        np.testing.assert_allclose(m, g * (1 - 0.9 ** t), rtol=1e-12)
        np.testing.assert_allclose(v, g * g * (1 - 0.999 ** t), rtol=1e-10)
    np.testing.assert_allclose(p, -50 * 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-9)


def test_adam_two_hand_computed_steps():
    # g1 = 0.5, g2 = -0.25, lr = 0.01, from p = 0:
    #  step 1: m = 0.05, v = 0.00025, m_hat = 0.5, v_hat = 0.25,
    #          p = -0.01 * 0.5 / (0.5 + 1e-8)
    #  step 2: m = 0.9*0.05 - 0.1*0.25 = 0.02,
    #          v = 0.999*0.00025 + 0.001*0.0625 = 0.00031225,
    #          m_hat = 0.02 / 0.19 = 2/19 (still positive: p keeps falling),
    #          v_hat = 0.00031225 / 0.001999
    p, m, v = mlp.adam_step([0.0], [0.5], [0.0], [0.0], 1, 0.01)
    assert abs(m[0] - 0.05) < 1e-15 * 0.05 and abs(v[0] - 0.00025) < 1e-14 * 0.00025
    p1 = -0.01 * 0.5 / (0.5 + 1e-8)
    assert abs(p[0] - p1) < 1e-15 * abs(p1)
    p, m, v = mlp.adam_step(p, [-0.25], m, v, 2, 0.01)
    assert abs(m[0] - 0.02) < 1e-14 * 0.02 and abs(v[0] - 0.00031225) < 1e-14 * 0.00031225
    want = p1 - 0.01 * (2 / 19) / (np.sqrt(0.00031225 / 0.001999) + 1e-8)
    assert abs(p[0] - want) < 1e-13 * abs(want)


def test_adam_matches_the_moving_average_sums():
    # m_t = (1 - b1) sum_i b1^(t-i) g_i and v_t = (1 - b2) sum_i b2^(t-i) g_i^2;
    # p_t = p_0 - sum_s lr * m_hat_s / (sqrt(v_hat_s) + eps)
    rng = np.random.default_rng(9)
    G = rng.normal(0, 1, (30, 16))
    p0 = rng.normal(0, 1, 16)
    p, m, v = p0.copy(), np.zeros(16), np.zeros(16)
    moved = np.zeros(16)
    for t in range(1, 31):
        p, m, v = mlp.adam_step(p, G[t - 1], m, v, t, 3e-3)
        w1 = 0.9 ** (t - np.arange(1, t + 1))
        w2 = 0.999 ** (t - np.arange(1, t + 1))
        ms = 0.1 * (w1 @ G[:t])
        vs = 0.001 * (w2 @ (G[:t] ** 2))
        np.testing.assert_allclose(m, ms, rtol=1e-11, atol=1e-14)
        np.testing.assert_allclose(v, vs, rtol=1e-11, atol=1e-16)
        moved += 3e-3 * (ms / (1 - 0.9 ** t)) / (np.sqrt(vs / (1 - 0.999 ** t)) + 1e-8)
    np.testing.assert_allclose(p, p0 - moved, rtol=1e-10, atol=1e-13)


def test_adam_is_invariant_to_the_gradient_scale():
    rng = np.random.default_rng(2)
    G = rng.normal(0, 1, (10, 8))
    pa = pb = rng.normal(0, 1, 8)
    ma = va = mb = vb = np.zeros(8)
    for t in range(1, 11):
        pa, ma, va = mlp.adam_step(pa, G[t - 1], ma, va, t, 1e-2)
        pb, mb, vb = mlp.adam_step(pb, 1000.0 * G[t - 1], mb, vb, t, 1e-2)
    np.testing.assert_allclose(pa, pb, rtol=1e-7, atol=1e-9)


# ---- the pins above reject plausible mistakes planted on the CPU -------------

def _adam_pins_hold(step):
    """The closed forms above, against any Adam implementation `step`."""
    g = np.array([0.5, -2.0, 7.0])
    p0 = np.array([0.1, 0.2, 0.3])
    p1, _, _ = step(p0, g, np.zeros(3), np.zeros(3), 1, 0.01)
    if not np.allclose(p1, p0 - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15):
        return False
    p, m, v = np.zeros(1), np.zeros(1), np.zeros(1)
    p, m, v = step(p, np.array([0.5]), m, v, 1, 0.01)
    p, m, v = step(p, np.array([-0.25]), m, v, 2, 0.01)
    want = -0.01 * 0.5 / (0.5 + 1e-8) - 0.01 * (2 / 19) / (np.sqrt(0.00031225 / 0.001999) + 1e-8)
    return abs(p[0] - want) < 1e-13 * abs(want)


def _bf16_pins_hold(fwd):
    return (fwd(_chain(w1=1 + 2 ** -7, b1=2 ** -9, b2=3 * 2 ** -10), _x(1.0))[0] == 1 + 2 ** -7
            and fwd(_chain(w2=1 + 2 ** -7, b2=2 ** -9), _x(1.0))[0] == 1 + 2 ** -7
            and fwd(_chain(b1=-2 ** -9), _x(1 + 2 ** -8 + 2 ** -10))[0] == 1 + 2 ** -7
            and fwd(_chain(w3=1 + 2 ** -8 + 2 ** -10), _x(1.0))[0] == 1 + 2 ** -7
            and fwd(_chain(w1=1 + 2 ** -7, b1=2 ** -9, b3=2 ** -12), _x(1.0))[0] == 1 + 2 ** -7 + 2 ** -12)


def test_pins_reject_planted_adam_mistakes():
    assert _adam_pins_hold(mlp.adam_step)

    def no_bias_correction(p, g, m, v, t, lr):
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        return p - lr * m / (np.sqrt(v) + 1e-8), m, v

    def betas_swapped(p, g, m, v, t, lr):
        return mlp.adam_step(p, g, m, v, t, lr, b1=0.999, b2=0.9)

    def eps_inside_sqrt(p, g, m, v, t, lr):
        m = 0.9 * m + 0.1 * g
        v = 0.999 * v + 0.001 * g * g
        return p - lr * (m / (1 - 0.9 ** t)) / np.sqrt(v / (1 - 0.999 ** t) + 1e-8), m, v

    def step_off_by_one(p, g, m, v, t, lr):
        return mlp.adam_step(p, g, m, v, t + 1, lr)

    for wrong in (no_bias_correction, betas_swapped, eps_inside_sqrt, step_off_by_one):
        assert not _adam_pins_hold(wrong), wrong.__name__


def test_pins_reject_planted_bf16_forward_mistakes():
    assert _bf16_pins_hold(mlp.forward_bf16)
    b = mlp.bf16

    def layers(p, X, r_x, r_h1, r_h2, r_y):
        w1, b1, w2, b2, w3, b3 = (b(np.asarray(a, dtype=np.float32)).astype(np.float64) for a in mlp.unpack(p))
        x = r_x(np.asarray(X, dtype=np.float32)).astype(np.float64)
        h1 = r_h1(np.maximum(x @ w1.T + b1, 0.0)).astype(np.float64)
        h2 = r_h2(np.maximum(h1 @ w2.T + b2, 0.0)).astype(np.float64)
        return r_y(h2 @ w3 + b3).astype(np.float64)

    same = lambda a: np.asarray(a, dtype=np.float64)  # noqa: E731

    def _unrounded_weights(p, X):
        w1, b1, w2, b2, w3, b3 = mlp.unpack(p)
        x = b(np.asarray(X, dtype=np.float32)).astype(np.float64)
        h1 = b(np.maximum(x @ w1.T + b1, 0.0)).astype(np.float64)
        h2 = b(np.maximum(h1 @ w2.T + b2, 0.0)).astype(np.float64)
        return h2 @ w3 + b3
    wrong = {
        "input not rounded": lambda p, X: layers(p, X, same, b, b, same),
        "h1 not rounded": lambda p, X: layers(p, X, b, same, b, same),
        "h2 not rounded": lambda p, X: layers(p, X, b, b, same, same),
        "output rounded": lambda p, X: layers(p, X, b, b, b, b),
        "weights not rounded": lambda p, X: _unrounded_weights(p, X),
        "plain FP64 forward": mlp.forward,
    }
    for name, fwd in wrong.items():
        assert not _bf16_pins_hold(fwd), name
