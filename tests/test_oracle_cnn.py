"""Pins of the CPU oracle of the refinement-flag predictor (oracle/cnn.py):
a textbook routine for the convolution, central finite differences for the
gradient, the naive formula for the loss, and convergence of Adam."""
import numpy as np
import pytest

from oracle import cnn

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv_single_channel_is_scipy_correlate2d():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(1, 1, 13, 17))
    w = rng.normal(size=(1, 1, 3, 3))
    b = np.array([0.25])
    y = cnn.conv(x, w, b)
    ref = scipy_signal.correlate2d(x[0, 0], w[0, 0], mode="same", boundary="fill", fillvalue=0.0) + 0.25
    assert np.allclose(y[0, 0], ref, rtol=0, atol=1e-12)


def test_conv_channels_sum_and_1x1():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 3, 6, 5))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = cnn.conv(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(scipy_signal.correlate2d(x[n, c], w[o, c], mode="same") for c in range(3))
            assert np.allclose(y[n, o], ref, atol=1e-12)
    w1 = rng.normal(size=(1, 3, 1, 1))
    y1 = cnn.conv(x, w1, np.zeros(1))
    assert np.allclose(y1[:, 0], np.einsum("c,nchw->nhw", w1[0, :, 0, 0], x), atol=1e-12)


def test_bce_matches_naive_formula():
    rng = np.random.default_rng(2)
    z = rng.normal(0, 3, size=(2, 7, 9))
    t = (rng.random(z.shape) < 0.4).astype(float)
    m = (rng.random(z.shape) < 0.8).astype(float)
    s = 1 / (1 + np.exp(-z))
    naive = -(t * np.log(s) + (1 - t) * np.log(1 - s))
    assert cnn.bce_loss(z, t, m) == pytest.approx((naive * m).sum() / m.sum(), rel=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    theta = cnn.init_params(5) * 0.7 + rng.normal(0, 0.05, cnn.n_params())
    x = rng.normal(size=(2, cnn.C_IN, 6, 7))
    t = (rng.random((2, 6, 7)) < 0.3).astype(float)
    m = (rng.random((2, 6, 7)) < 0.9).astype(float)
    loss, g = cnn.backward(theta, x, t, m)
    assert loss == pytest.approx(cnn.bce_loss(cnn.forward(theta, x)[0], t, m), rel=1e-14)
    idx = rng.choice(cnn.n_params(), 60, replace=False)
    eps = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (cnn.bce_loss(cnn.forward(tp, x)[0], t, m) - cnn.bce_loss(cnn.forward(tm, x)[0], t, m)) / (2 * eps)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_adam_minimises_a_quadratic():
    target = np.array([1.0, -2.0, 0.5])
    th = np.zeros(3)
    m = np.zeros(3)
    v = np.zeros(3)
    for t in range(1, 3001):
        g = 2 * (th - target)
        th, m, v = cnn.adam_step(th, g, m, v, t, lr=1e-2)
    assert np.abs(th - target).max() < 1e-3


def test_features_zero_outside_cover_and_on_dry_cells():
    h = np.array([[2.0, 0.0005], [1.0, 3.0]])
    B = np.array([[-2.0, 0.3], [-1.1, -2.5]])
    cov = np.array([[True, True], [True, False]])
    f = cnn.features(h, h * 0.1, h * 0.2, B, cov, np.array([[1, 0], [0, 1]]))
    assert f[0, 0, 1] == 0.0 and f[:, 1, 1].sum() == 0.0
    assert f[0, 1, 0] == pytest.approx((1.0 - 1.1) / 0.1)
    assert f[4, 0, 0] == 1.0 and f[4, 1, 1] == 0.0
