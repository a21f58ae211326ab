"""CPU FP64 oracle of the warm-start network's building blocks (test infrastructure only;
see mca_oracle for the rules).  Plain NumPy definitions:

* conv2d(x, w, b, d): y[n,co,p] = b[co] + sum_ci sum_(ky,kx) w[co,ci,ky,kx]
  x[n,ci, p + d*(ky-r, kx-r)], r = (K-1)/2, with zero padding (output size = input size),
  for a K x K kernel (K odd);
* leaky ReLU with slope 0.1;
* the analytic gradients of the convolution with respect to x, w and b;
* mean squared error and one Adam step (Kingma & Ba, bias-corrected).
"""
from __future__ import annotations

import numpy as np


def _shifted(x, dy, dx):
    """x[..., y + dy, x + dx] with zeros outside."""
    H, W = x.shape[-2:]
    out = np.zeros_like(x)
    if abs(dy) >= H or abs(dx) >= W:        # the shifted window lies wholly in the padding
        return out
    ys = slice(max(0, -dy), min(H, H - dy))
    xs = slice(max(0, -dx), min(W, W - dx))
    yt = slice(max(0, dy), min(H, H + dy))
    xt = slice(max(0, dx), min(W, W + dx))
    out[..., ys, xs] = x[..., yt, xt]
    return out


def conv2d(x, w, b, d):
    N, Cin, H, W = x.shape
    Cout, _, K, _ = w.shape
    r = (K - 1) // 2
    y = np.broadcast_to(b[None, :, None, None], (N, Cout, H, W)).astype(np.float64).copy()
    for ky in range(K):
        for kx in range(K):
            xs = _shifted(x, d * (ky - r), d * (kx - r))
            y += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xs)
    return y


def leaky(z):
    return np.where(z > 0, z, 0.1 * z)


def conv2d_backward(x, w, d, gz):
    """Gradients of L with respect to x, w, b given gz = dL/dz of z = conv2d(x, w, b, d)."""
    K = w.shape[-1]
    r = (K - 1) // 2
    gx = np.zeros_like(x, dtype=np.float64)
    gw = np.zeros_like(w, dtype=np.float64)
    for ky in range(K):
        for kx in range(K):
            dy, dx = d * (ky - r), d * (kx - r)
            xs = _shifted(x, dy, dx)
            gw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", gz, xs)
            gx += _shifted(np.einsum("oc,nohw->nchw", w[:, :, ky, kx], gz), -dy, -dx)
    gb = gz.sum(axis=(0, 2, 3))
    return gx, gw, gb


def mse(pred, target):
    r = pred - target
    return float(np.mean(r * r)), 2.0 * r / r.size


def adam_step(w, g, m, v, lr, b1, b2, eps, t):
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
