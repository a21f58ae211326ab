"""Pins of the CNN oracle: the convolution against SciPy's 2-D correlation, and its
analytic gradients against central finite differences."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn_oracle as C


@pytest.mark.parametrize("d", [1, 2, 3])
def test_conv_matches_scipy_correlate(d):
    rng = np.random.default_rng(d)
    x = rng.standard_normal((2, 3, 9, 11))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = C.conv3x3(x, w, b, d)
    for n in range(2):
        for co in range(4):
            ref = np.full((9, 11), b[co])
            for ci in range(3):
                k = np.zeros((2 * d + 1, 2 * d + 1))
                k[::d, ::d] = w[co, ci]          # dilated kernel
                ref += correlate2d(x[n, ci], k, mode="same", boundary="fill")
            np.testing.assert_allclose(y[n, co], ref, rtol=1e-12, atol=1e-12)


def test_conv_gradients_finite_difference():
    rng = np.random.default_rng(4)
    d = 2
    x = rng.standard_normal((2, 2, 6, 7))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    gy = rng.standard_normal((2, 3, 6, 7))

    def loss(x_, w_, b_):
        return float(np.sum(C.leaky(C.conv3x3(x_, w_, b_, d)) * gy))

    y = C.leaky(C.conv3x3(x, w, b, d))
    gz = gy * np.where(y > 0, 1.0, 0.1)
    gx, gw, gb = C.conv3x3_backward(x, w, d, gz)
    h = 1e-6
    for arr, grad in ((x, gx), (w, gw), (b, gb)):
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, size=min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp = loss(x, w, b)
            flat[idx] = old - h
            lm = loss(x, w, b)
            flat[idx] = old
            np.testing.assert_allclose(grad.reshape(-1)[idx], (lp - lm) / (2 * h), rtol=1e-5,
                                       atol=1e-7)


def test_mse_and_adam_closed_forms():
    p = np.array([1.0, 2.0, 4.0])
    t = np.array([1.0, 1.0, 1.0])
    loss, g = C.mse(p, t)
    assert loss == pytest.approx((0 + 1 + 9) / 3)
    np.testing.assert_allclose(g, 2 * (p - t) / 3)
    # first Adam step moves every weight by lr * sign(g) (bias correction cancels)
    w, m, v = C.adam_step(np.zeros(3), np.array([0.5, -2.0, 1e-3]), np.zeros(3), np.zeros(3),
                          1e-2, 0.9, 0.999, 1e-12, 1)
    np.testing.assert_allclose(w, -1e-2 * np.array([1.0, -1.0, 1.0]), rtol=1e-6)
