"""Warm-start network kernels against the CPU oracle through the C ABI: the tensor-core
convolution forward and backward (data and weight gradients, with ragged pixel tiles, 3 x 3
and 11 x 11 kernels and dilations), loss, Adam, the BF16 operand tiles, features, targets
and guesses; a short training run; the fallback rule of the warm-started solve; and the
trained network's effect on the solve at 256^2, 512^2 and 1024^2.

Tolerances: BF16 operands are rounded on the host the way the kernels round them (to
nearest even), so the products are exact and only the FP32 accumulation differs from the
FP64 oracle: within 1e-5 of the sum of the magnitudes of the terms (K^2 x 32 products
per output of the forward pass, every pixel of the images per weight gradient)."""
import os

import numpy as np
import pytest

import mca_inputs as mi
from oracle import cnn_oracle as C
from oracle import mca_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_07929_gb300 as mca  # noqa: E402
from paper_2109_07929_gb300 import cnn  # noqa: E402

DEV = "cuda:0"


def _bf16(a):
    """Nearest BF16 (ties to even) of the FP32 values, as float64 (the kernels' rounding)."""
    t = torch.as_tensor(np.asarray(a, np.float32))
    return t.to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)


def _nhwc(x_nchw):
    """NCHW values -> NHWC32 BF16 device tensor (int16 bit patterns), channels padded."""
    N, Cc, H, W = x_nchw.shape
    t = torch.zeros(N, H, W, 32, dtype=torch.float32)
    t[..., :Cc] = torch.as_tensor(np.transpose(x_nchw, (0, 2, 3, 1)), dtype=torch.float32)
    return t.to(torch.bfloat16).view(torch.int16).to(DEV)


def _from_nhwc(t, Cc):
    x = t.view(torch.bfloat16).to(torch.float32).cpu().numpy().astype(np.float64)
    return np.transpose(x[..., :Cc], (0, 3, 1, 2))


def _tiles(w):
    """Forward and backward BF16 tiles of master weights w[cout][cin][K][K] (library kernel)."""
    cout, cin, K, _ = w.shape
    cm = 16 if cout <= 16 else 32
    wd = torch.as_tensor(np.asarray(w, np.float32), device=DEV)
    wf = torch.empty(K * K, cm, 32, dtype=torch.int16, device=DEV)
    wb = torch.empty(K * K, 32, 32, dtype=torch.int16, device=DEV)
    assert mca.load().mca_cnn_prep_weights(wd.data_ptr(), cout, cin, K, cm, wf.data_ptr(),
                                           wb.data_ptr(), None) == 0
    return wf, wb, cm


CASES = [  # (N, cin, cout, H, W, K, d, act)
    (2, 5, 11, 9, 150, 3, 1, 1),
    (1, 4, 32, 7, 130, 11, 1, 1),
    (2, 32, 32, 12, 40, 11, 3, 0),
    (1, 32, 2, 5, 260, 11, 2, 0),
]


@pytest.mark.parametrize("N,cin,cout,H,W,K,d,act", CASES)
def test_conv_forward_and_backward_match_oracle(N, cin, cout, H, W, K, d, act):
    lib = mca.load()
    rng = np.random.default_rng(H * W + K)
    x = _bf16(rng.standard_normal((N, cin, H, W)))
    w = _bf16(rng.standard_normal((cout, cin, K, K)) / np.sqrt(cin * K * K))
    b = rng.standard_normal(cout).astype(np.float32).astype(np.float64)
    z = C.conv2d(x, w, b, d)
    y_ref = C.leaky(z) if act else z
    wf, wb, cm = _tiles(w)
    xd = _nhwc(x)
    out = torch.empty(N, H, W, 32, dtype=torch.int16, device=DEV)
    out32 = torch.empty(N, H, W, cout, dtype=torch.float32, device=DEV)
    bd = torch.as_tensor(b.astype(np.float32), device=DEV)
    assert lib.mca_cnn_conv(xd.data_ptr(), N, H, W, wf.data_ptr(), K, d, cm, cout, bd.data_ptr(),
                            act, 0, None, out.data_ptr(), out32.data_ptr(), None) == 0
    assert lib.mca_cnn_check(None) == 0
    # FP32 accumulation of exact BF16 products: 1e-5 of the summed term magnitudes
    scale = C.conv2d(np.abs(x), np.abs(w), np.abs(b), d)
    y32 = np.transpose(out32.cpu().numpy(), (0, 3, 1, 2))
    assert np.all(np.abs(y32 - y_ref) <= 1e-5 * scale + 1e-30)
    ybf = _from_nhwc(out, cout)
    assert np.all(np.abs(ybf - y_ref) <= 2.0 ** -8 * np.abs(y_ref) + 1e-5 * scale)
    assert np.all(out.view(torch.bfloat16)[..., cout:].cpu().float().numpy() == 0)

    # backward data: dL/dx of the layer from gz, times the leaky-ReLU derivative of yprev
    if cin > 32 or N * H * W > 5000:
        return
    gz = _bf16(rng.standard_normal((N, cout, H, W)))
    yprev = _bf16(rng.standard_normal((N, cin, H, W)))
    gx_ref, gw_ref, gb_ref = C.conv2d_backward(x, w, d, gz)
    gx_ref = gx_ref * np.where(yprev > 0, 1.0, 0.1)
    gzd, ypd = _nhwc(gz), _nhwc(yprev)
    gx = torch.empty(N, H, W, 32, dtype=torch.int16, device=DEV)
    gx32 = torch.empty(N, H, W, cin, dtype=torch.float32, device=DEV)
    assert lib.mca_cnn_conv(gzd.data_ptr(), N, H, W, wb.data_ptr(), K, d, 32, cin, None, 1, 1,
                            ypd.data_ptr(), gx.data_ptr(), gx32.data_ptr(), None) == 0
    gscale = np.abs(C.conv2d_backward(np.ones_like(x), np.abs(w), d, np.abs(gz))[0])
    g32 = np.transpose(gx32.cpu().numpy(), (0, 3, 1, 2))
    assert np.all(np.abs(g32 - gx_ref) <= 1e-5 * gscale + 1e-30)
    # weight and bias gradients (tensor cores, MN-major operands)
    nf = int(lib.mca_cnn_wgrad_scratch(N, H, W, K))
    scratch = torch.empty(nf, dtype=torch.float32, device=DEV)
    gw = torch.empty(cout, cin, K, K, dtype=torch.float32, device=DEV)
    gb = torch.empty(cout, dtype=torch.float32, device=DEV)
    assert lib.mca_cnn_conv_wgrad(xd.data_ptr(), gzd.data_ptr(), N, H, W, K, d, cin, cout,
                                  scratch.data_ptr(), gw.data_ptr(), gb.data_ptr(), None) == 0
    assert lib.mca_cnn_check(None) == 0
    wscale = C.conv2d_backward(np.abs(x), np.abs(w), d, np.abs(gz))[1]
    assert np.all(np.abs(gw.cpu().numpy() - gw_ref) <= 1e-5 * wscale + 1e-30)
    np.testing.assert_allclose(gb.cpu().numpy(), gb_ref, rtol=1e-5,
                               atol=1e-5 * np.abs(gz).sum(axis=(0, 2, 3)).max())


def test_loss_adam_features_targets_and_guess():
    lib = mca.load()
    rng = np.random.default_rng(3)
    npix = 1000
    p = rng.standard_normal((npix, 2)).astype(np.float32)
    t = rng.standard_normal((npix, 2)).astype(np.float32)
    loss_ref, g_ref = C.mse(p.astype(np.float64), t.astype(np.float64))
    pd, td = torch.as_tensor(p, device=DEV), torch.as_tensor(t, device=DEV)
    gz = torch.empty(npix, 32, dtype=torch.int16, device=DEV)
    part = torch.empty(256, dtype=torch.float32, device=DEV)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    assert lib.mca_cnn_loss(pd.data_ptr(), td.data_ptr(), npix, gz.data_ptr(), part.data_ptr(),
                            loss.data_ptr(), None) == 0
    assert float(loss.item()) == pytest.approx(loss_ref, rel=1e-5)
    g = gz.view(torch.bfloat16).float().cpu().numpy()
    np.testing.assert_array_equal(g[:, :2], _bf16(g_ref.astype(np.float32)))
    assert np.all(g[:, 2:] == 0)
    # Adam against the oracle's step
    w0, gr = rng.standard_normal(64), rng.standard_normal(64).astype(np.float32)
    w, m, v = w0.copy(), np.zeros(64), np.zeros(64)
    wd = torch.as_tensor(w0.astype(np.float32), device=DEV)
    gd = torch.as_tensor(gr, device=DEV)
    md, vd = torch.zeros_like(wd), torch.zeros_like(wd)
    for step in (1, 2, 3):
        w, m, v = C.adam_step(w, gr.astype(np.float64), m, v, 1e-2, 0.9, 0.999, 1e-8, step)
        assert lib.mca_cnn_adam(wd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), 64,
                                1e-2, 0.9, 0.999, 1e-8, step, None) == 0
    np.testing.assert_allclose(wd.cpu().numpy(), w, rtol=1e-5, atol=1e-6)
    # features, targets, guesses (two crossbars in one batch through a map index)
    m_, n_ = 12, 17
    cbs = [mi.make_crossbar(m_, n_, s) for s in (4, 5)]
    gm = torch.as_tensor(np.stack([c.gmap for c in cbs]), device=DEV)
    vin = torch.as_tensor(np.concatenate([c.vin for c in cbs]), device=DEV)
    mp = torch.as_tensor(np.array([1, 0], np.int32), device=DEV)
    vlt = torch.as_tensor(rng.uniform(0, 0.3, (2, m_, n_)), device=DEV)
    vlb = torch.as_tensor(rng.uniform(0, 0.05, (2, m_, n_)), device=DEV)
    model = cnn.WarmStartCNN(seed=1)
    x = model.features(torch.flip(gm, [0]), mp, vin, vlt, vlb, m_, n_)
    xf = x.view(torch.bfloat16).float().cpu().numpy()
    for k in range(2):
        np.testing.assert_array_equal(xf[k, ..., 0], _bf16(np.log10(cbs[k].gmap) + 5))
        np.testing.assert_array_equal(xf[k, ..., 1],
                                      _bf16(np.repeat(cbs[k].vin[0][:, None] / cnn.VSCALE, n_, 1)))
        np.testing.assert_array_equal(xf[k, ..., 2], _bf16(vlt[k].cpu().numpy() / cnn.VSCALE))
        np.testing.assert_array_equal(xf[k, ..., 3],
                                      _bf16(vlb[k].cpu().numpy() * cnn.BSCALE / cnn.VSCALE))
    assert np.all(xf[..., 4:] == 0)
    vst = vlt + 1e-4
    vsb = vlb - 2e-4
    tg = model.targets(vst, vsb, vlt, vlb, m_, n_).cpu().numpy()
    np.testing.assert_allclose(tg[..., 0], 1e-4 * cnn.DSCALE, rtol=1e-4)
    np.testing.assert_allclose(tg[..., 1], -2e-4 * cnn.DSCALE, rtol=1e-4)
    st = model.state(torch.as_tensor(tg, device=DEV), vlt, vlb, m_, n_).cpu().numpy()
    np.testing.assert_allclose(st[:, :m_ * n_].reshape(2, m_, n_), vst.cpu().numpy(), rtol=1e-9,
                               atol=1e-10)
    np.testing.assert_allclose(st[:, m_ * n_:].reshape(2, m_, n_), vsb.cpu().numpy(), rtol=1e-9,
                               atol=1e-10)
    st0 = model.state(None, vlt, vlb, m_, n_).cpu().numpy()
    np.testing.assert_array_equal(st0[:, :m_ * n_].reshape(2, m_, n_), vlt.cpu().numpy())


def test_short_training_reduces_loss():
    model = cnn.WarmStartCNN(seed=2)
    losses, _, _ = cnn.train(model, samples=64, size=64, batch=8, epochs=6, lr=2e-3,
                             seed0=7_000_000, log=lambda *a: None)
    assert losses[-1] < 0.7 * losses[0]


def test_warm_start_solve_keeps_the_better_start():
    """Newton from the guess or from the fallback state (V_lin), whichever has the smaller
    KCL residual, always to the tolerance: exact solutions are kept, NaN guesses and a
    guess worse than V_lin are replaced by V_lin."""
    cb = mi.make_crossbar(40, 56, 8, nvec=3)
    p = cb.params
    kw = dict(g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot, g_src=p.g_src,
              g_term_top_right=p.g_term_top_right, g_term_bot_top=p.g_term_bot_top,
              g_sense=p.g_sense, b=p.b, max_batch=3)
    model = cnn.WarmStartCNN(seed=3)
    v = torch.as_tensor(cb.vin, device=DEV)
    with mca.Solver(mca.default_params(40, 56, newton_rtol=1e-11, **kw), cb.gmap) as s, \
            mca.Solver(mca.default_params(40, 56, max_newton=1, **kw), cb.gmap) as s1:
        vt0, vb0, _, st0 = s.solve(cb.vin)
        vlt = torch.empty(3, 40, 56, dtype=torch.float64, device=DEV)
        vlb = torch.empty_like(vlt)
        s1.solve(v, vlt, vlb, allow_not_converged=True)
        vlin = model.state(None, vlt, vlb, 40, 56)
        exact = torch.as_tensor(np.concatenate([vt0.reshape(3, -1), vb0.reshape(3, -1)], 1),
                                device=DEV)
        worse = vlin + 1e-3
        bad = torch.full_like(exact, float("nan"))
        runs = [s.solve_from(v, g_, fallback=vlin) for g_ in (exact, worse, bad)]
    for k in range(3):
        ref = O.newton_solve(p, cb.gmap, cb.vin[k], tol=1e-13, linear="direct")
        for vt, vb, _, st in runs:
            assert st[k]["status"] == 0
            assert np.abs(vt[k] - ref.Vt).max() / np.abs(ref.Vt).max() < 1e-7
            assert np.abs(vb[k] - ref.Vb).max() / np.abs(ref.Vb).max() < 1e-7
        assert runs[0][3][k]["fallback"] == 0 and runs[0][3][k]["newton_iters"] <= 1
        assert runs[1][3][k]["fallback"] == 1 and runs[2][3][k]["fallback"] == 1


@pytest.mark.skipif(not os.path.exists(cnn.WEIGHTS), reason="trained weights not present")
def test_trained_network_effect_on_the_solve():
    """The committed trained network on held-out crossbars at 256^2 (the training size),
    512^2 and 1024^2: every warm-started solve reaches 1e-8 and the bookkeeping of the warm
    path (first Newton step, network, Newton from the accepted start) is consistent; the
    figures (iterations saved, fallback rate, residual ratio of the guess over V_lin, time)
    are printed."""
    model = cnn.WarmStartCNN(seed=0).load()
    for size, count in ((256, 4), (512, 2), (1024, 1)):
        r = cnn.evaluate(model, size, count, log=print)
        assert r["max_residual_base"] <= 1e-8 and r["max_residual_warm"] <= 1e-8
        assert 0.0 <= r["fallback_rate"] <= 1.0
        assert r["newton_warm"] >= 1.0 and r["gmres_warm"] >= 1.0
        assert r["residual_ratio_guess_over_vlin"]["min"] > 0.0
