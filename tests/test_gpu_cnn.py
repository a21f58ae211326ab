"""Warm-start network kernels against the CPU oracle (forward, gradients, loss, Adam,
feature/state conversion), a short training run, and the warm-started solve, whose
result must not depend on the guess."""
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


def _bf16_round(a):
    """Round FP32 values to the nearest BF16 (ties to even) and return them as float64."""
    b = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _bits(a):
    return torch.as_tensor((np.asarray(a, np.float32).view(np.uint32) >> 16).astype(np.uint16)
                           .view(np.int16), device=DEV)


def _f32(a):
    return torch.as_tensor(np.asarray(a, np.float32), device=DEV)


@pytest.mark.parametrize("d,act", [(1, 1), (3, 0), (2, 1)])
def test_conv_forward_and_backward_match_oracle(d, act):
    lib = mca.load()
    rng = np.random.default_rng(d + 10 * act)
    N, Cin, Cout, H, W = 2, 5, 11, 9, 13
    x = rng.standard_normal((N, Cin, H, W)).astype(np.float32).astype(np.float64)
    w = _bf16_round(rng.standard_normal((Cout, Cin, 3, 3)) * 0.3)
    b = rng.standard_normal(Cout).astype(np.float32).astype(np.float64)
    gy = rng.standard_normal((N, Cout, H, W)).astype(np.float32).astype(np.float64)
    z = C.conv3x3(x, w, b, d)
    y_ref = C.leaky(z) if act else z
    gz = gy * (np.where(y_ref > 0, 1.0, 0.1) if act else 1.0)
    gx_ref, gw_ref, gb_ref = C.conv3x3_backward(x, w, d, gz)

    xd, yd = _f32(x), torch.empty(N, Cout, H, W, dtype=torch.float32, device=DEV)
    wb, bd = _bits(w), _f32(b)
    assert lib.mca_cnn_conv_forward(xd.data_ptr(), N, Cin, H, W, wb.data_ptr(), bd.data_ptr(),
                                    Cout, d, act, yd.data_ptr(), None) == 0
    np.testing.assert_allclose(yd.cpu().numpy(), y_ref, rtol=2e-5, atol=2e-5)
    gyd = _f32(gy)
    gzs = torch.empty_like(yd)
    gx = torch.empty_like(xd)
    gw = torch.empty(Cout, Cin, 3, 3, dtype=torch.float32, device=DEV)
    gb = torch.empty(Cout, dtype=torch.float32, device=DEV)
    nchunk = 7
    part = torch.empty(nchunk * (Cout * Cin * 9 + Cout), dtype=torch.float32, device=DEV)
    assert lib.mca_cnn_conv_backward(xd.data_ptr(), yd.data_ptr(), gyd.data_ptr(), N, Cin, H, W,
                                     wb.data_ptr(), Cout, d, act, gzs.data_ptr(), gx.data_ptr(),
                                     gw.data_ptr(), gb.data_ptr(), part.data_ptr(), nchunk,
                                     None) == 0
    torch.cuda.synchronize()
    np.testing.assert_allclose(gx.cpu().numpy(), gx_ref, rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(gw.cpu().numpy(), gw_ref, rtol=1e-4, atol=1e-3)
    np.testing.assert_allclose(gb.cpu().numpy(), gb_ref, rtol=1e-4, atol=1e-4)


def test_mse_and_adam_match_oracle():
    lib = mca.load()
    rng = np.random.default_rng(3)
    p, t = rng.standard_normal(1000), rng.standard_normal(1000)
    loss_ref, g_ref = C.mse(p.astype(np.float32).astype(np.float64),
                            t.astype(np.float32).astype(np.float64))
    pd, td = _f32(p), _f32(t)
    g = torch.empty_like(pd)
    part = torch.empty(256, dtype=torch.float32, device=DEV)
    loss = torch.empty(1, dtype=torch.float32, device=DEV)
    assert lib.mca_cnn_mse(pd.data_ptr(), td.data_ptr(), 1000, g.data_ptr(), part.data_ptr(),
                           loss.data_ptr(), None) == 0
    assert float(loss.item()) == pytest.approx(loss_ref, rel=1e-5)
    np.testing.assert_allclose(g.cpu().numpy(), g_ref, rtol=1e-5)
    w0, gr = rng.standard_normal(64), rng.standard_normal(64)
    w, m, v = w0.copy(), np.zeros(64), np.zeros(64)
    wd, gd = _f32(w0), _f32(gr)
    md, vd = torch.zeros_like(wd), torch.zeros_like(wd)
    for step in (1, 2, 3):
        w, m, v = C.adam_step(w, gr.astype(np.float32).astype(np.float64), m, v, 1e-2, 0.9,
                              0.999, 1e-8, step)
        assert lib.mca_cnn_adam(wd.data_ptr(), None, gd.data_ptr(), md.data_ptr(), vd.data_ptr(),
                                64, 1e-2, 0.9, 0.999, 1e-8, step, None) == 0
    np.testing.assert_allclose(wd.cpu().numpy(), w, rtol=1e-5, atol=1e-6)


def test_features_and_state_conversion():
    cb = mi.make_crossbar(12, 17, 4, nvec=2)
    model = cnn.WarmStartCNN(seed=1)
    g = torch.as_tensor(cb.gmap, device=DEV)
    v = torch.as_tensor(cb.vin, device=DEV)
    x = model.features(g, v, 12, 17).cpu().numpy()
    np.testing.assert_allclose(x[:, 0], np.broadcast_to(np.log10(cb.gmap) + 5, (2, 12, 17)),
                               rtol=1e-6)
    np.testing.assert_allclose(x[1, 1], np.repeat(cb.vin[1][:, None] / cnn.VSCALE, 17, 1),
                               rtol=1e-6)
    np.testing.assert_allclose(x[0, 2, 3], np.arange(17) / 16, rtol=1e-6)
    np.testing.assert_allclose(x[0, 3, :, 5], np.arange(12) / 11, rtol=1e-6)
    st = torch.as_tensor(np.random.default_rng(0).uniform(0, 0.3, (2, 2 * 12 * 17)), device=DEV)
    y = model.targets(st, 12, 17)
    lib = mca.load()
    back = torch.empty_like(st)
    assert lib.mca_cnn_state(y.data_ptr(), back.data_ptr(), 2, 12, 17, cnn.VSCALE, cnn.BSCALE, 1,
                             None, None) == 0
    np.testing.assert_allclose(back.cpu().numpy(), st.cpu().numpy(), rtol=1e-6)


def test_short_training_reduces_loss():
    X, T, G, V = cnn.make_dataset(32, size=48, seed0=7_000_000, group=16, log=lambda *a: None)
    model = cnn.WarmStartCNN(seed=2)
    l0 = float(model.train_step(X[:8].contiguous(), T[:8].contiguous(), 8, 48, 48, 0.0).item())
    losses, _ = cnn.train(model, X, T, epochs=12, batch=8, lr=3e-3, log=lambda *a: None)
    assert losses[-1] < 0.5 * l0


def test_warm_start_solve_is_judged_by_newton():
    cb = mi.make_crossbar(40, 56, 8, nvec=3)
    p = cb.params
    params = mca.default_params(40, 56, g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot,
                                g_src=p.g_src, g_term_top_right=p.g_term_top_right,
                                g_term_bot_top=p.g_term_bot_top, g_sense=p.g_sense, b=p.b,
                                newton_rtol=1e-11, max_batch=3)
    model = cnn.WarmStartCNN(seed=3)                     # untrained: arbitrary guesses
    g = torch.as_tensor(cb.gmap, device=DEV)
    v = torch.as_tensor(cb.vin, device=DEV)
    with mca.Solver(params, cb.gmap) as s:
        vt0, vb0, _, st0 = s.solve(cb.vin)
        guess = model.guess(g, v, 40, 56)
        vt1, vb1, _, st1 = s.solve_from(v, guess)
        exact = torch.as_tensor(np.concatenate([vt0.reshape(3, -1), vb0.reshape(3, -1)], 1),
                                device=DEV)
        vt2, vb2, _, st2 = s.solve_from(v, exact)
        bad = torch.full_like(exact, float("nan"))
        vt3, vb3, _, st3 = s.solve_from(v, bad)
    for k in range(3):
        ref = O.newton_solve(p, cb.gmap, cb.vin[k], tol=1e-13, linear="direct")
        for vt, vb, st in ((vt1, vb1, st1), (vt2, vb2, st2), (vt3, vb3, st3)):
            assert st[k]["status"] == 0
            assert np.abs(vt[k] - ref.Vt).max() / np.abs(ref.Vt).max() < 1e-7
            assert np.abs(vb[k] - ref.Vb).max() / np.abs(ref.Vb).max() < 1e-7
        assert st2[k]["fallback"] == 0 and st2[k]["newton_iters"] <= 1
        assert st3[k]["fallback"] == 1
