"""Pins of the FP64 warm-start network reference (oracle/cnn_oracle.py) against things other
than itself: brute-force loops for the convolution, central finite differences for every
gradient, closed forms for the loss and for Adam's first steps."""
import numpy as np
import pytest

from oracle import cnn_oracle as C
from paper_2509_18544_gb300 import synth


def brute_conv(x, W, b):
    n, c, h, w = x.shape
    o = W.shape[0]
    ho, wo = (h + 1) // 2, (w + 1) // 2
    z = np.zeros((n, o, ho, wo))
    for a in range(n):
        for k in range(o):
            for i in range(ho):
                for j in range(wo):
                    s = b[k]
                    for ci in range(c):
                        for u in range(3):
                            for v in range(3):
                                yy, xx = 2 * i + u - 1, 2 * j + v - 1
                                if 0 <= yy < h and 0 <= xx < w:
                                    s += W[k, ci, u, v] * x[a, ci, yy, xx]
                    z[a, k, i, j] = s
    return z


@pytest.mark.parametrize("h,w", [(6, 6), (5, 7)])
def test_conv_forward_matches_loops(h, w):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, h, w))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    assert np.allclose(C.conv_forward(x, W, b), brute_conv(x, W, b), rtol=1e-13, atol=1e-13)


def test_conv_backward_matches_finite_differences():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 3, 6, 5))
    W = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    gz = rng.normal(size=(2, 4, 3, 3))
    L = lambda x_, W_, b_: float(np.sum(gz * C.conv_forward(x_, W_, b_)))
    gx, gW, gb = C.conv_backward(x, W, gz)
    eps = 1e-6
    for arr, g in ((x, gx), (W, gW), (b, gb)):
        flat = arr.reshape(-1)
        for k in rng.choice(flat.size, min(12, flat.size), replace=False):
            old = flat[k]
            flat[k] = old + eps
            lp = L(x, W, b)
            flat[k] = old - eps
            lm = L(x, W, b)
            flat[k] = old
            assert abs((lp - lm) / (2 * eps) - g.reshape(-1)[k]) <= 1e-7 * (1 + abs(g.reshape(-1)[k]))


def test_mse_closed_form():
    y = np.array([[1.0, 2.0], [3.0, 5.0]])
    t = np.array([[0.0, 2.0], [1.0, 1.0]])
    loss, g = C.mse(y, t)
    assert loss == pytest.approx((1 + 0 + 4 + 16) / 4)
    assert np.allclose(g, 2 * (y - t) / 4)


def test_network_gradients_match_finite_differences():
    n_out = 7
    rng = np.random.default_rng(3)
    p = synth.cnn_init(n_out, seed=5).astype(np.float64)
    p += 0.01 * rng.normal(size=p.size)          # non-zero biases, so every term is exercised
    x = rng.random((2, 18, 32, 32))
    t = rng.normal(size=(2, n_out))
    loss, g, gx = C.gradients(p, x, t, n_out)
    f = lambda q, xx: C.mse(C.forward(q, xx, n_out)[0], t)[0]
    assert loss == pytest.approx(f(p, x), rel=1e-14)
    eps = 1e-6
    # a sample of parameters from every layer, and of input pixels
    bounds = np.cumsum([0] + [int(np.prod(s)) for s in C.param_shapes(n_out)])
    idx = np.concatenate([rng.integers(bounds[i], bounds[i + 1], 4) for i in range(len(bounds) - 1)])
    for k in idx:
        q = p.copy()
        q[k] += eps
        lp = f(q, x)
        q[k] -= 2 * eps
        lm = f(q, x)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(abs(g[k]), 1e-3 * np.abs(g).max()), (k, fd, g[k])
    for flat in rng.choice(x.size, 8, replace=False):
        xx = x.copy().reshape(-1)
        xx[flat] += eps
        lp = f(p, xx.reshape(x.shape))
        xx[flat] -= 2 * eps
        lm = f(p, xx.reshape(x.shape))
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gx.reshape(-1)[flat]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(gx).max())


def test_relu_gradient_is_zero_where_inactive():
    # a network whose first-layer biases switch every unit off has zero gradients upstream
    n_out = 3
    p = synth.cnn_init(n_out, seed=1).astype(np.float64)
    P = C.unflatten(p, n_out)
    P[1][:] = -1e6
    p2 = C.flatten(P)
    x = np.random.default_rng(0).random((1, 18, 32, 32))
    _, g, gx = C.gradients(p2, x, np.ones((1, n_out)), n_out)
    assert np.all(g[:int(np.prod(C.param_shapes(n_out)[0])) + 32] == 0)
    assert np.all(gx == 0)


def test_adam_first_steps_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g1 = np.array([0.3, -4.0, 1e-3])
    m = v = np.zeros(3)
    p1, m, v = C.adam_step(p, g1, m, v, 1, lr=0.01)
    # first step: mhat = g, vhat = g^2, so the move is lr g / (|g| + eps)
    assert np.allclose(p1, p - 0.01 * g1 / (np.abs(g1) + 1e-8), rtol=1e-15)
    g2 = np.array([0.1, 1.0, -1e-3])
    p2, m2, v2 = C.adam_step(p1, g2, m, v, 2, lr=0.01)
    mh = (0.9 * 0.1 * g1 + 0.1 * g2) / (1 - 0.81)
    vh = (0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2) / (1 - 0.999 ** 2)
    assert np.allclose(p2, p1 - 0.01 * mh / (np.sqrt(vh) + 1e-8), rtol=1e-14)


def test_parameter_layout():
    n_out = 726
    assert C.param_count(n_out) == synth.cnn_init(n_out, 0).size == 126614
    shapes = C.param_shapes(n_out)
    assert shapes[0] == (32, 18, 3, 3) and shapes[-2] == (726, 128)
