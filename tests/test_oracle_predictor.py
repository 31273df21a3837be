"""Pins of the oracle's predictor MLP (12 -> 64 -> 64 -> 1, Sec. 7.1 with an MLP):
parameter count, forward pass against a numpy composition, gradients against
central finite differences, and the closed form of Adam's first step."""
import numpy as np


def _theta(orc, seed=0, scale=0.3):
    return np.random.default_rng(seed).standard_normal(orc.pred_nparams()) * scale


def _unpack(th):
    o = 0
    W1 = th[o:o + 768].reshape(64, 12); o += 768
    b1 = th[o:o + 64]; o += 64
    W2 = th[o:o + 4096].reshape(64, 64); o += 4096
    b2 = th[o:o + 64]; o += 64
    W3 = th[o:o + 64].reshape(1, 64); o += 64
    b3 = th[o:o + 1]
    return W1, b1, W2, b2, W3, b3


def test_param_count(orc):
    assert orc.pred_nparams() == 12 * 64 + 64 + 64 * 64 + 64 + 64 + 1 == 5057


def test_forward_matches_numpy(orc):
    th = _theta(orc)
    X = np.random.default_rng(1).standard_normal((33, 12))
    W1, b1, W2, b2, W3, b3 = _unpack(th)
    h = np.maximum(X @ W1.T + b1, 0)
    h = np.maximum(h @ W2.T + b2, 0)
    ref = (h @ W3.T + b3)[:, 0]
    np.testing.assert_allclose(orc.pred_forward(th, X), ref, rtol=1e-12, atol=1e-12)


def test_gradient_central_differences(orc):
    th = _theta(orc, 2)
    g0 = np.random.default_rng(3)
    X = g0.standard_normal((17, 12))
    t = g0.standard_normal(17)
    loss, g = orc.pred_grad(th, X, t)
    y = orc.pred_forward(th, X)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-12 * max(1, loss)
    idx = g0.choice(th.size, 300, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        fd = (orc.pred_grad(tp, X, t)[0] - orc.pred_grad(tm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, np.abs(g).max()), (i, fd, g[i])


def test_adam_first_step_closed_form(orc):
    th = _theta(orc, 4)
    g = np.random.default_rng(5).standard_normal(th.size)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    th1 = th.copy()
    orc.adam_step(th1, g, m, v, 1, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8)
    # bias-corrected first moments equal g and g^2: step = lr * g / (|g| + eps)
    np.testing.assert_allclose(th1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m, (1 - 0.9) * g, rtol=1e-15)
    np.testing.assert_allclose(v, (1 - 0.999) * g * g, rtol=1e-15)


def test_training_reduces_loss(orc):
    g0 = np.random.default_rng(6)
    X = g0.standard_normal((256, 12))
    t = np.sin(X[:, 0]) + 0.5 * X[:, 1] ** 2
    th = _theta(orc, 7, 0.1)
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    l0 = orc.pred_grad(th, X, t)[0]
    for step in range(1, 301):
        _, g = orc.pred_grad(th, X, t)
        orc.adam_step(th, g, m, v, step, lr=3e-3)
    assert orc.pred_grad(th, X, t)[0] < 0.2 * l0
