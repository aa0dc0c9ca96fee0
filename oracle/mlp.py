"""FP64 oracle of the learned switch's cost model (TEST INFRASTRUCTURE ONLY).

The model is a plain two-hidden-layer perceptron, 12 -> 64 (ReLU) -> 64
(ReLU) -> 1, trained on the mean squared error.  Parameters are one flat
array laid out W1[64][12] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3.
This module is the definition written out in NumPy (forward, the analytic
gradient, a BF16-rounding forward for the inference path, and one Adam
update); the tests pin the gradient against central finite differences of
the forward, the BF16 forward against a hand-set network whose rounded and
unrounded outputs differ by a hand-derived amount, and the Adam update
against the closed forms of its moving averages.
"""
import numpy as np

IN, HID = 12, 64
W1, B1 = 0, HID * IN
W2 = B1 + HID
B2 = W2 + HID * HID
W3 = B2 + HID
B3 = W3 + HID
NPARAMS = B3 + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    return (p[W1:B1].reshape(HID, IN), p[B1:W2], p[W2:B2].reshape(HID, HID), p[B2:W3], p[W3:B3], p[B3])


def forward(p, X):
    w1, b1, w2, b2, w3, b3 = unpack(p)
    h1 = np.maximum(np.asarray(X, dtype=np.float64) @ w1.T + b1, 0.0)
    h2 = np.maximum(h1 @ w2.T + b2, 0.0)
    return h2 @ w3 + b3


def loss(p, X, T):
    e = forward(p, X) - np.asarray(T, dtype=np.float64)
    return float(np.mean(e * e))


def loss_grad(p, X, T):
    """Returns (L, dL/dp) by the chain rule, written layer by layer."""
    w1, b1, w2, b2, w3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    a1 = X @ w1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ w2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ w3 + b3
    e = y - np.asarray(T, dtype=np.float64)
    L = float(np.mean(e * e))
    dy = 2.0 * e / n
    g = np.zeros(NPARAMS)
    g[W3:B3] = h2.T @ dy
    g[B3] = dy.sum()
    da2 = np.outer(dy, w3) * (a2 > 0)
    g[W2:B2] = (da2.T @ h1).reshape(-1)
    g[B2:W3] = da2.sum(axis=0)
    da1 = (da2 @ w2) * (a1 > 0)
    g[W1:B1] = (da1.T @ X).reshape(-1)
    g[B1:W2] = da1.sum(axis=0)
    return L, g


def bf16(x):
    """Round FP32 values to BF16 (round to nearest, ties to even), as FP32."""
    b = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def forward_bf16(p, X):
    """Inference as the in-loop decision computes it: BF16 weights, inputs and
    hidden activations; sums carried in higher precision."""
    w1, b1, w2, b2, w3, b3 = (bf16(np.asarray(a, dtype=np.float32)).astype(np.float64) for a in unpack(p))
    x = bf16(np.asarray(X, dtype=np.float32)).astype(np.float64)
    h1 = bf16(np.maximum(x @ w1.T + b1, 0.0)).astype(np.float64)
    h2 = bf16(np.maximum(h1 @ w2.T + b2, 0.0)).astype(np.float64)
    return h2 @ w3 + b3


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(p, g, m, v, t, lr, b1=ADAM_B1, b2=ADAM_B2, eps=ADAM_EPS):
    """One Adam update (Kingma & Ba, "Adam: A Method for Stochastic
    Optimization", Algorithm 1), in FP64, for step number t >= 1:
    the first and second moment estimates are exponential moving averages of
    the gradient and of its square, each divided by (1 - beta^t) to undo
    their bias towards the zero start, and the parameters move by
    lr * m_hat / (sqrt(v_hat) + eps).  Returns (p, m, v) after the step."""
    assert t >= 1
    g = np.asarray(g, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1 ** t)
    v_hat = v / (1.0 - b2 ** t)
    p = np.asarray(p, dtype=np.float64) - lr * m_hat / (np.sqrt(v_hat) + eps)
    return p, m, v
