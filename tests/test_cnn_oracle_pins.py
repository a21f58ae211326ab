"""Pins of the CNN oracle: the convolution against SciPy's 2-D correlation (3 x 3, 5 x 5 and
11 x 11 kernels, dilated), and its analytic gradients against central finite differences."""
import numpy as np
import pytest
from scipy.signal import correlate2d

from oracle import cnn_oracle as C


@pytest.mark.parametrize("K,d", [(3, 1), (3, 2), (3, 3), (5, 2), (11, 1), (11, 3)])
def test_conv_matches_scipy_correlate(K, d):
    rng = np.random.default_rng(d + K)
    span = d * (K - 1) + 1
    H, W = max(9, span + 2), max(11, span + 5)     # the dilated kernel fits the image
    x = rng.standard_normal((2, 3, H, W))
    w = rng.standard_normal((4, 3, K, K))
    b = rng.standard_normal(4)
    y = C.conv2d(x, w, b, d)
    for n in range(2):
        for co in range(4):
            ref = np.full((H, W), b[co])
            for ci in range(3):
                k = np.zeros((span, span))
                k[::d, ::d] = w[co, ci]          # dilated kernel
                ref += correlate2d(x[n, ci], k, mode="same", boundary="fill")
            np.testing.assert_allclose(y[n, co], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("K,d,H,W", [(5, 2, 3, 4), (3, 4, 2, 9), (11, 3, 4, 5)])
def test_conv_matches_loop_definition_beyond_the_image(K, d, H, W):
    """Dilated kernels wider than the image: every tap outside it reads the zero padding
    (the definition y[n,co,i,j] = b[co] + sum w[co,ci,ky,kx] x[n,ci,i+d(ky-r),j+d(kx-r)],
    x = 0 outside), written as plain loops."""
    rng = np.random.default_rng(K * d)
    x = rng.standard_normal((1, 2, H, W))
    w = rng.standard_normal((3, 2, K, K))
    b = rng.standard_normal(3)
    r = (K - 1) // 2
    ref = np.zeros((1, 3, H, W))
    for co in range(3):
        for i in range(H):
            for j in range(W):
                s = b[co]
                for ci in range(2):
                    for ky in range(K):
                        for kx in range(K):
                            yy, xx = i + d * (ky - r), j + d * (kx - r)
                            if 0 <= yy < H and 0 <= xx < W:
                                s += w[co, ci, ky, kx] * x[0, ci, yy, xx]
                ref[0, co, i, j] = s
    np.testing.assert_allclose(C.conv2d(x, w, b, d), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("K,d", [(3, 2), (5, 1)])
def test_conv_gradients_finite_difference(K, d):
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 2, 6, 7))
    w = rng.standard_normal((3, 2, K, K))
    b = rng.standard_normal(3)
    gy = rng.standard_normal((2, 3, 6, 7))

    def loss(x_, w_, b_):
        return float(np.sum(C.leaky(C.conv2d(x_, w_, b_, d)) * gy))

    y = C.leaky(C.conv2d(x, w, b, d))
    gz = gy * np.where(y > 0, 1.0, 0.1)
    gx, gw, gb = C.conv2d_backward(x, w, d, gz)
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
