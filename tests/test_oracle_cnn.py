"""Pins of the oracle CNN: conv3d against scipy's correlate, gradients against
central finite differences in float64, Adam against its closed form."""
import numpy as np
import pytest
from scipy.signal import correlate

from oracle import cnn


def test_conv3d_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    b = rng.standard_normal(2)
    y = cnn.conv3d(x, w, b)
    for o in range(2):
        ref = b[o] + sum(correlate(x[c], w[o, c], mode="same", method="direct") for c in range(3))
        assert np.allclose(y[o], ref, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    layers = ((4, 5), (5, 3))
    params = cnn.init_params(3, layers)
    params = [(w, rng.standard_normal(b.shape) * 0.1) for w, b in params]
    x = rng.standard_normal((4, 4, 5, 3))
    t = rng.standard_normal((3, 4, 5, 3))
    out, acts = cnn.forward(params, x)
    L, grads = cnn.backward(params, acts, t)
    h = 1e-6
    for li in range(2):
        for q in range(2):
            arr = params[li][q]
            flat = arr.reshape(-1)
            for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + h
                lp = cnn.loss(cnn.forward(params, x)[0], t)
                flat[idx] = old - h
                lm = cnn.loss(cnn.forward(params, x)[0], t)
                flat[idx] = old
                fd = (lp - lm) / (2 * h)
                an = grads[li][q].reshape(-1)[idx]
                assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (li, q, idx, fd, an)


def test_input_gradient_of_conv_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((2, 3, 4, 5))
    w = rng.standard_normal((3, 2, 3, 3, 3))
    dy = rng.standard_normal((3, 3, 4, 5))
    dx, _, _ = cnn.conv3d_backward(x, w, dy)
    f = lambda xx: float(np.sum(cnn.conv3d(xx, w, np.zeros(3)) * dy))
    h = 1e-6
    for idx in rng.choice(x.size, 8, replace=False):
        xp = x.copy().reshape(-1); xp[idx] += h
        xm = x.copy().reshape(-1); xm[idx] -= h
        fd = (f(xp.reshape(x.shape)) - f(xm.reshape(x.shape))) / (2 * h)
        assert abs(fd - dx.reshape(-1)[idx]) <= 1e-7 * max(1, abs(fd))


def test_adam_first_step_moves_by_lr_times_sign():
    # closed form: after one step m_hat = g, v_hat = g^2, so the update is lr * g / (|g| + eps)
    params = [(np.array([[1.0, -2.0]]), np.array([0.5]))]
    grads = [(np.array([[3.0, -0.5]]), np.array([1e-3]))]
    new = cnn.adam_step(params, grads, {}, lr=0.1)
    assert np.allclose(new[0][0], [[0.9, -1.9]], atol=1e-6)
    assert np.allclose(new[0][1], [0.4], atol=1e-4)
