"""GPU parity of every step of the solve against the CPU FP64 oracle, through the C ABI.

Tolerances:
* FP64 kernels (residual, Jacobian apply, eigenpairs, FP64 preconditioner, GMRES): FP64
  rounding, scaled by the magnitude of the terms that cancel.
* Whole solves: relative KCL residual <= the requested tolerance (recomputed here by the
  oracle's own residual) and node-voltage max relative error <= 1e-7 against the oracle
  solution, both solved tight.
* Tensor-core preconditioner: BF16 operands (unit roundoff 2^-9) with FP32 accumulation;
  the forward transforms carry a relative error of a few 1e-3 in the mode coefficients,
  so z agrees with the FP64 oracle to 3e-2 in relative 2-norm (a transposed or misplaced
  tile gives O(1) errors).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import mca_inputs as mi
from oracle import mca_oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2109_07929_gb300 as mca  # noqa: E402

DEV = "cuda:0"


def _params(p, **kw):
    base = dict(g_wire_top=p.g_wire_top, g_wire_bot=p.g_wire_bot, g_src=p.g_src,
                g_term_top_right=p.g_term_top_right, g_term_bot_top=p.g_term_bot_top,
                g_sense=p.g_sense, b=p.b, neg_ratio=p.neg_ratio,
                device_model=mca.DEVICE_YAKOPCIC if p.neg_ratio != 1.0 else mca.DEVICE_SINH)
    base.update(kw)
    return mca.default_params(p.rows, p.cols, **base)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _rel_err(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


SHAPES = [(1, 1), (1, 9), (7, 1), (33, 47), (64, 64), (130, 70)]

# D = g cosh(b dV) (eq. J) is evaluated in FP32 where |b dV| < 3/4.  Relative error budget,
# in units of 2^-24: g rounded to FP32 (1); coshf, 2 ulp of a value in [1, 1.3) (4); the
# FP32 argument, dV rounded once and times b rounded once, through |x| tanh|x| < 0.48 (1);
# the product g cosh (1); for the Yakopcic form the FP32 amplitude and its product (2).
# In all 9 x 2^-24 = 5.4e-7.
D_RTOL = 5.5e-7


@pytest.mark.parametrize("m,n", SHAPES + [(257, 129)])
def test_eigenpairs(m, n):
    cb = mi.make_crossbar(m, n, 1, g_wire_bot=0.5)
    with mca.Solver(_params(cb.params, precision=mca.PREC_FP64, max_batch=1), cb.gmap) as s:
        mu, qr, nu, qc = s.eigenpairs()
    mu_r, qr_r, nu_r, qc_r = O.eig_setup(cb.params)
    for lam, Q, lam_r, Q_r in ((mu, qr, mu_r, qr_r), (nu, qc, nu_r, qc_r)):
        k = lam.size
        np.testing.assert_allclose(lam, lam_r, rtol=0, atol=5e-15 * np.abs(lam_r).max())
        sign = np.sign(np.sum(Q * Q_r, axis=0))
        np.testing.assert_allclose(Q * sign[None, :], Q_r, atol=1e-9)
        np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-10)


@pytest.mark.parametrize("vrange", [0.35, 2.0], ids=["series", "wide"])
@pytest.mark.parametrize("m,n", SHAPES)
def test_residual_and_jacobian_diagonal(m, n, vrange):
    """|b dV| < 3/4 uses the economised polynomial for sinh, larger |b dV| the library function;
    both must give the residual to FP64 rounding.  D (cosh, the Jacobian diagonal) is
    evaluated in FP32: it only shapes the Newton matrix."""
    cb = mi.make_crossbar(m, n, 2, nvec=2)
    p = cb.params
    rng = np.random.default_rng(5)
    x = rng.uniform(-vrange / 3.5, vrange, size=(2, 2 * m * n))
    with mca.Solver(_params(p, precision=mca.PREC_FP64, max_batch=2), cb.gmap) as s:
        F = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
        D = torch.empty(2, m * n, dtype=torch.float64, device=DEV)
        fn, dm = s.residual(_t(x), _t(cb.vin), F, D)
        F = F.cpu().numpy()
        D = D.cpu().numpy()
    Gt, Gb = O.layer_operators(p)
    for v in range(2):
        Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], x[v, :m * n], x[v, m * n:])
        dv = x[v, :m * n] - x[v, m * n:]
        cur = np.abs(cb.gmap.ravel() / p.b * np.sinh(p.b * dv)).max()
        scale = 4 * max(p.g_wire_top, p.g_wire_bot) * np.abs(x[v]).max() + p.g_src * 0.3 + cur
        np.testing.assert_allclose(F[v], np.concatenate([Ft, Fb]), rtol=0, atol=1e-14 * scale)
        Dr = O.device_conductance(cb.gmap.ravel(), p.b, x[v, :m * n] - x[v, m * n:])
        np.testing.assert_allclose(D[v], Dr, rtol=D_RTOL)
        np.testing.assert_allclose(fn[v], np.linalg.norm(np.concatenate([Ft, Fb])), rtol=1e-12)
        np.testing.assert_allclose(dm[v], Dr.mean(), rtol=3e-7)


def _term_sizes(p, gmap, vin, Vt, Vb, neg_ratio=1.0):
    """Per-entry sum of the absolute values of the terms of eq. (F): |G| |x| for the wire
    operators (diagonal and couplings), the device current and the source current."""
    Gt, Gb = O.layer_operators(p)
    cur = np.abs(O.device_current(gmap.ravel(), p.b, Vt - Vb, neg_ratio))
    Yt, _ = O.source_vector(p, vin)
    st = abs(Gt) @ np.abs(Vt) + cur + np.abs(Yt)
    sb = abs(Gb) @ np.abs(Vb) + cur
    return np.concatenate([st, sb])


@pytest.mark.parametrize("neg_ratio", [1.0, 0.35], ids=["sinh", "yakopcic"])
@pytest.mark.parametrize("vrange", [0.35, 2.0], ids=["series", "wide"])
@pytest.mark.parametrize("m,n", SHAPES + [(256, 256), (37, 700), (3, 1024), (1100, 640)])
def test_residual_pair(m, n, vrange, neg_ratio):
    """The FP32-pair residual against eq. (F): each entry within 2^-42 of the size of its
    terms (an exact-arithmetic model of the cell peaks at 2^-44.6 on these inputs), ||F||
    within the bound the call returns, that bound at most 2^-40 of the sizes' 2-norm, and
    D and mean(D) as from mca_residual.  "wide" states reach the library branch of sinh.
    The four larger shapes take the column-strip walk with shared-memory staging (37 x 700
    and 1100 x 640: a ragged last strip and block ranges that cross strips; 3 x 1024: one
    row per block; 1100 x 640: about five rows per block, so the bottom layer's rows roll
    through registers), the small shapes the per-cell loop."""
    cb = mi.make_crossbar(m, n, 2, nvec=2, neg_ratio=neg_ratio)
    p = cb.params
    rng = np.random.default_rng(15)
    x = rng.uniform(-vrange / 3.5, vrange, size=(2, 2 * m * n))
    # voltages the split takes through its general path (zeros, |x| < 2^-74) among
    # ordinary ones
    special = np.array([0.0, -0.0, 1e-30, -2e-23, 3e-22, 1e-5, -7e-3])
    x[1, ::7] = special[np.arange(x[1, ::7].size) % special.size]
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=2), cb.gmap) as s:
        F = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
        D = torch.empty(2, m * n, dtype=torch.float64, device=DEV)
        fn, dm, fe = s.residual_pair(_t(x), _t(cb.vin), F, D)
        F = F.cpu().numpy()
        D = D.cpu().numpy()
    for v in range(2):
        vt, vb = x[v, :m * n], x[v, m * n:]
        Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], vt, vb)
        ref = np.concatenate([Ft, Fb])
        size = _term_sizes(p, cb.gmap, cb.vin[v], vt, vb, neg_ratio)
        err = np.abs(F[v] - ref)
        assert (err <= 2.0 ** -42 * size + 2.0 ** -96).all(), (err / size).max()
        assert abs(fn[v] - np.linalg.norm(ref)) <= fe[v]
        assert fe[v] <= 2.0 ** -40 * np.linalg.norm(size) * 1.001
        Dr = O.device_conductance(cb.gmap.ravel(), p.b, vt - vb, neg_ratio)
        np.testing.assert_allclose(D[v], Dr, rtol=D_RTOL)
        np.testing.assert_allclose(dm[v], Dr.mean(), rtol=3e-7)


def test_residual_pair_needs_fp32_tail():
    cb = mi.make_crossbar(8, 8, 1, b=0.001)
    with mca.Solver(_params(cb.params, precision=mca.PREC_BF16_SPLIT, max_batch=1),
                    cb.gmap) as s:
        x = _t(np.zeros((1, 128)))
        F = torch.empty(1, 128, dtype=torch.float64, device=DEV)
        D = torch.empty(1, 64, dtype=torch.float64, device=DEV)
        with pytest.raises(RuntimeError):
            s.residual_pair(x, _t(cb.vin), F, D)


def test_pair_residual_hands_convergence_to_fp64():
    """The pair residual never decides convergence.  A warm start from converged solutions
    takes the pair residual first (no linear solve yet), finds ||F|| within 10x of the target
    and must hand each vector to the FP64 residual: two residual launches for zero Newton
    steps, and the oracle confirms the states.  A cold solve at 1e-8 takes the FP64 residual
    directly after its last linear solve (launches = Newton steps + 1)."""
    cb = mi.make_crossbar(48, 40, 3, nvec=2)
    p = cb.params
    N = 48 * 40
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, newton_rtol=1e-8, max_batch=2),
                    cb.gmap) as s:
        s.profile(True)
        vt, vb, io, st = s.solve(cb.vin)
        cold = s.profile_read()["residual"]["launches"]
        s.profile(False)
        s.profile(True)
        guess = np.concatenate([vt.reshape(2, N), vb.reshape(2, N)], axis=1)
        vt2, vb2, io2, st2 = s.solve_from(cb.vin, _t(guess))
        warm = s.profile_read()["residual"]["launches"]
    assert cold == max(st[v]["newton_iters"] for v in range(2)) + 1
    assert warm == 2
    for v in range(2):
        assert st2[v]["status"] == 0 and st2[v]["newton_iters"] == 0, st2[v]
        Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], vt2[v].ravel(), vb2[v].ravel())
        Yt, _ = O.source_vector(p, cb.vin[v])
        assert np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt) <= 1e-8 * 1.01


@pytest.mark.parametrize("b", [0.01, 5000.0])
def test_residual_outside_fp32_tail_range(b):
    """b = 0.01 and b = 5000 put the polynomial's folded tail coefficients outside the FP32
    range the kernel allows, so the whole polynomial runs in FP64; both branches of
    |b dV| < 3/4 are hit.  Same bar as above."""
    m, n = 40, 37
    cb = mi.make_crossbar(m, n, 21, nvec=2, b=b)
    p = cb.params
    rng = np.random.default_rng(22)
    x = rng.uniform(-0.3 / b, 1.2 / b, size=(2, 2 * m * n))
    with mca.Solver(_params(p, precision=mca.PREC_FP64, max_batch=2), cb.gmap) as s:
        F = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
        D = torch.empty(2, m * n, dtype=torch.float64, device=DEV)
        s.residual(_t(x), _t(cb.vin), F, D)
        F = F.cpu().numpy()
        D = D.cpu().numpy()
    for v in range(2):
        dv = x[v, :m * n] - x[v, m * n:]
        assert (np.abs(b * dv) < 0.75).any() and (np.abs(b * dv) > 0.75).any()
        Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], x[v, :m * n], x[v, m * n:])
        cur = np.abs(cb.gmap.ravel() / p.b * np.sinh(p.b * dv)).max()
        scale = 4 * max(p.g_wire_top, p.g_wire_bot) * np.abs(x[v]).max() + p.g_src * 0.3 + cur
        np.testing.assert_allclose(F[v], np.concatenate([Ft, Fb]), rtol=0, atol=1e-14 * scale)
        Dr = O.device_conductance(cb.gmap.ravel(), p.b, dv)
        np.testing.assert_allclose(D[v], Dr, rtol=D_RTOL)


@pytest.mark.parametrize("m,n", [(1, 1), (33, 47), (130, 70)])
def test_yakopcic_residual_and_jacobian_diagonal(m, n):
    """Yakopcic-form devices (a2/a1 = 0.35) under both polarities: the residual to FP64
    rounding and the Jacobian diagonal to the FP32 conductance tolerance."""
    cb = mi.make_crossbar(m, n, 4, nvec=2, neg_ratio=0.35)
    p = cb.params
    rng = np.random.default_rng(8)
    x = rng.uniform(-0.3, 0.3, size=(2, 2 * m * n))
    with mca.Solver(_params(p, precision=mca.PREC_FP64, max_batch=2), cb.gmap) as s:
        F = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
        D = torch.empty(2, m * n, dtype=torch.float64, device=DEV)
        fn, dm = s.residual(_t(x), _t(cb.vin), F, D)
        F = F.cpu().numpy()
        D = D.cpu().numpy()
    for v in range(2):
        dv = x[v, :m * n] - x[v, m * n:]
        assert (dv < 0).any() or m * n == 1
        Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], x[v, :m * n], x[v, m * n:])
        cur = np.abs(O.device_current(cb.gmap.ravel(), p.b, dv, p.neg_ratio)).max()
        scale = 4 * max(p.g_wire_top, p.g_wire_bot) * np.abs(x[v]).max() + p.g_src * 0.3 + cur
        np.testing.assert_allclose(F[v], np.concatenate([Ft, Fb]), rtol=0, atol=1e-14 * scale)
        Dr = O.device_conductance(cb.gmap.ravel(), p.b, dv, p.neg_ratio)
        np.testing.assert_allclose(D[v], Dr, rtol=D_RTOL)
        np.testing.assert_allclose(dm[v], Dr.mean(), rtol=3e-7)


@pytest.mark.parametrize("prec", [mca.PREC_FP64, mca.PREC_BF16_SPLIT], ids=["fp64", "bf16split"])
@pytest.mark.parametrize("m,n", [(1, 1), (48, 40)])
def test_yakopcic_solve_signed_inputs(m, n, prec):
    """Newton on Yakopcic-form devices (a2/a1 = 0.5) with inputs of both signs, against
    the oracle's direct-solve Newton."""
    cb = mi.make_crossbar(m, n, 19, nvec=3, vmin=-0.3, neg_ratio=0.5)
    assert (cb.vin < 0).any()
    _check_solve(cb, prec, 1e-10)


@pytest.mark.parametrize("m,n", SHAPES)
def test_jacobian_apply(m, n):
    cb = mi.make_crossbar(m, n, 3)
    p = cb.params
    rng = np.random.default_rng(6)
    xt = rng.uniform(0, 0.3, size=m * n)
    xb = rng.uniform(0, 0.1, size=m * n)
    z = rng.standard_normal((2, 2 * m * n))
    Dr = O.device_conductance(cb.gmap.ravel(), p.b, xt - xb)
    J = O.jacobian(p, cb.gmap, xt, xb)
    with mca.Solver(_params(p, precision=mca.PREC_FP64, max_batch=2), cb.gmap) as s:
        w = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
        s.jacobian_apply(_t(np.stack([Dr, Dr])), _t(z), w)
        w = w.cpu().numpy()
    for v in range(2):
        ref = J @ z[v]
        np.testing.assert_allclose(w[v], ref, rtol=0, atol=1e-14 * 8 * np.abs(z[v]).max())


@pytest.mark.parametrize("wires", ["unit", "odd"])
@pytest.mark.parametrize("m,n", SHAPES + [(256, 256)])
def test_jacobian_apply_fp32_z(m, n, wires):
    """w = J z with FP32 z in the three arithmetics of the solver, against the definition,
    each row's error relative to the size of its terms (|J| |z|): the FP32-pair form within
    2^-44 (a few roundings of its low parts, each 2^-48 of the terms; an exact-arithmetic
    model of these inputs peaks at 2^-45.9), the FP64 form within 2^-50 (five FP64
    roundings), the FP32 form within 2^-20 (eight FP32 roundings, constants included).  "odd" wire and
    termination conductances are not FP32 numbers, so their low halves are exercised; half
    of the D values are FP32 numbers (as from the FP32 conductance) and half are not.  The
    second vector is smooth (neighbours nearly equal), where the wire terms cancel to a few
    parts in 1e4 of their size."""
    kw = {} if wires == "unit" else dict(g_wire_top=0.7, g_wire_bot=0.3, g_src=1.3,
                                         g_term_top_right=1e-3 / 3, g_term_bot_top=1e-3 / 7,
                                         g_sense=1.1)
    cb = mi.make_crossbar(m, n, 9, **kw)
    p = cb.params
    rng = np.random.default_rng(12)
    xt = rng.uniform(0, 0.3, size=m * n)
    xb = rng.uniform(0, 0.1, size=m * n)
    Dr = O.device_conductance(cb.gmap.ravel(), p.b, xt - xb)
    Dr[::2] = Dr[::2].astype(np.float32).astype(np.float64)
    Gt, Gb = O.layer_operators(p)
    Dm = sp.diags(Dr)
    J = sp.bmat([[Gt + Dm, -Dm], [-Dm, Gb + Dm]], format="csr")
    z = np.empty((2, 2 * m * n), dtype=np.float32)
    z[0] = rng.standard_normal(2 * m * n)
    ii, jj = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    smooth = np.sin(0.01 * ii + 0.013 * jj).ravel()
    z[1] = np.concatenate([smooth, 0.5 * smooth]) * (1 + 1e-4 * rng.standard_normal(2 * m * n))
    z64 = z.astype(np.float64)
    # per-row size of the terms of J z: |diag z_i| + sum |offdiag z_j|
    Jabs = np.abs(J)
    out = {}
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=2), cb.gmap) as s:
        Dd = _t(np.stack([Dr, Dr]))
        zd = torch.as_tensor(z, device=DEV)
        for mode in (mca.APPLY_PAIR, mca.APPLY_F64, mca.APPLY_F32):
            w = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
            s.jacobian_apply_f32(Dd, zd, w, mode=mode)
            out[mode] = w.cpu().numpy()
    for v in range(2):
        ref = J @ z64[v]
        size = Jabs @ np.abs(z64[v])
        for mode, bound in ((mca.APPLY_PAIR, 2.0 ** -44), (mca.APPLY_F64, 2.0 ** -50),
                            (mca.APPLY_F32, 2.0 ** -20)):
            err = np.abs(out[mode][v] - ref)
            assert (err <= bound * size).all(), (mode, v, (err / np.maximum(size, 1e-300)).max())
    # the cancellation case separates the forms: relative to the result itself, the
    # FP32 form is far off where the pair form is not
    ref = J @ z64[1]
    if m * n > 1:
        rel = lambda w: np.linalg.norm(w - ref) / np.linalg.norm(ref)  # noqa: E731
        assert rel(out[mca.APPLY_PAIR][1]) < 1e-11
        assert rel(out[mca.APPLY_F32][1]) > 100 * rel(out[mca.APPLY_PAIR][1])


def test_jacobian_apply_fp32_z_rejects_bad_mode():
    cb = mi.make_crossbar(8, 8, 1)
    with mca.Solver(_params(cb.params, precision=mca.PREC_BF16_SPLIT, max_batch=1),
                    cb.gmap) as s:
        D = _t(np.ones((1, 64)))
        z = torch.zeros(1, 128, dtype=torch.float32, device=DEV)
        w = torch.empty(1, 128, dtype=torch.float64, device=DEV)
        with pytest.raises(RuntimeError):
            s.jacobian_apply_f32(D, z, w, mode=7)


@pytest.mark.parametrize("m,n", SHAPES + [(256, 256)])
def test_precond_fp64(m, n):
    cb = mi.make_crossbar(m, n, 4, g_wire_bot=0.5)
    p = cb.params
    rng = np.random.default_rng(7)
    r = rng.standard_normal((2, 2 * m * n))
    a = np.array([2.1e-5, 7.0e-5])
    eig = O.eig_setup(p)
    with mca.Solver(_params(p, precision=mca.PREC_FP64, max_batch=2), cb.gmap) as s:
        z = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
        s.precond_apply(a, _t(r), z)
        z = z.cpu().numpy()
    for v in range(2):
        zt, zb = O.precond_apply_modes(eig, a[v], a[v], r[v, :m * n], r[v, m * n:], (m, n))
        ref = np.concatenate([zt, zb])
        assert _rel_err(z[v], ref) < 1e-9


@pytest.mark.parametrize("prec", [mca.PREC_BF16, mca.PREC_BF16_SPLIT], ids=["bf16", "bf16split"])
@pytest.mark.parametrize("m,n", [(1, 1), (33, 47), (128, 128), (130, 70), (256, 384)])
def test_precond_tensor_core(m, n, prec):
    cb = mi.make_crossbar(m, n, 4, g_wire_bot=0.5)
    p = cb.params
    rng = np.random.default_rng(8)
    r = rng.standard_normal((3, 2 * m * n))
    a = np.array([2.1e-5, 7.0e-5, 3.3e-4])
    eig = O.eig_setup(p)
    with mca.Solver(_params(p, precision=prec, max_batch=3), cb.gmap) as s:
        z = torch.empty(3, 2 * m * n, dtype=torch.float64, device=DEV)
        s.precond_apply(a, _t(r), z)
        z = z.cpu().numpy()
    for v in range(3):
        zt, zb = O.precond_apply_modes(eig, a[v], a[v], r[v, :m * n], r[v, m * n:], (m, n))
        ref = np.concatenate([zt, zb])
        err = np.linalg.norm(z[v] - ref) / np.linalg.norm(ref)
        assert err < 3e-2, (v, err)


@pytest.mark.parametrize("m,n", [(1, 1), (33, 47), (130, 70), (256, 256)])
def test_precond_mhat_paper_form(m, n):
    """The paper's own evaluation (eq. block with M_hat, tridiagonal solves) against the
    oracle's literal evaluation of the same formulas."""
    cb = mi.make_crossbar(m, n, 4, g_wire_bot=0.5)
    p = cb.params
    rng = np.random.default_rng(7)
    r = rng.standard_normal((2, 2 * m * n))
    a = np.array([2.1e-5, 7.0e-5])
    with mca.Solver(_params(p, precision=mca.PREC_MHAT, max_batch=2), cb.gmap) as s:
        z = torch.empty(2, 2 * m * n, dtype=torch.float64, device=DEV)
        s.precond_apply(a, _t(r), z)
        z = z.cpu().numpy()
    for v in range(2):
        z1, z2 = O.precond_apply_block(p, None, a[v], a[v], r[v, :m * n], r[v, m * n:],
                                       minv=lambda w: O.mhat_apply_inverse(p, a[v], a[v], w))
        assert _rel_err(z[v], np.concatenate([z1, z2])) < 1e-8


@pytest.mark.parametrize("prec", [mca.PREC_FP64, mca.PREC_BF16_SPLIT], ids=["fp64", "bf16split"])
def test_gmres_cycle(prec):
    cb = mi.make_crossbar(40, 56, 9)
    p = cb.params
    m, n = p.rows, p.cols
    N = m * n
    rng = np.random.default_rng(3)
    xt = rng.uniform(0, 0.3, N)
    xb = rng.uniform(0, 0.05, N)
    J = O.jacobian(p, cb.gmap, xt, xb)
    Dr = O.device_conductance(cb.gmap.ravel(), p.b, xt - xb)
    a = Dr.mean()
    rhs = rng.standard_normal(2 * N)
    with mca.Solver(_params(p, precision=prec, max_batch=1), cb.gmap) as s:
        dx = torch.empty(1, 2 * N, dtype=torch.float64, device=DEV)
        its, res = s.gmres_solve(_t(Dr[None]), [a], _t(rhs[None]), dx, 1e-9)   # one cycle
        dx = dx.cpu().numpy()[0]
    true_res = np.linalg.norm(rhs - J @ dx)
    assert true_res <= 1.5e-9 * np.linalg.norm(rhs)
    np.testing.assert_allclose(res[0], true_res, rtol=1e-3, atol=1e-13 * np.linalg.norm(rhs))
    eig = O.eig_setup(p)
    pc = lambda v: np.concatenate(O.precond_apply_modes(eig, a, a, v[:N], v[N:], (m, n)))
    _, its_ref, _ = O.gmres_right(lambda v: J @ v, rhs, pc, restart=30, rtol=1e-9)
    if prec == mca.PREC_FP64:
        assert abs(int(its[0]) - its_ref) <= 1
    else:
        assert its[0] <= its_ref + 4


def _check_solve(cb, prec, tol, vtol=1e-7, nvec=None, ref_tol=1e-13):
    p = cb.params
    vin = cb.vin if nvec is None else cb.vin[:nvec]
    with mca.Solver(_params(p, precision=prec, newton_rtol=tol, max_batch=min(4, len(vin))),
                    cb.gmap) as s:
        vt, vb, io, st = s.solve(vin)
    for v in range(len(vin)):
        assert st[v]["status"] == 0, st[v]
        Ft, Fb = O.residual(p, cb.gmap, vin[v], vt[v].ravel(), vb[v].ravel())
        Yt, _ = O.source_vector(p, vin[v])
        rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
        assert rel <= tol * 1.01, (v, rel)
        np.testing.assert_allclose(st[v]["rel_residual"], rel, rtol=1e-3, atol=tol * 1e-3)
        ref = O.newton_solve(p, cb.gmap, vin[v], tol=ref_tol, linear="direct")
        if prec == mca.PREC_FP64:
            # the FP64 form: max relative error per layer
            assert _rel_err(vt[v], ref.Vt) <= vtol and _rel_err(vb[v], ref.Vb) <= vtol
        else:
            # mixed-precision forms: errors on the scale of the solution (both layers), which
            # is what the KCL stop test bounds; a layer far below the other (the bottom node
            # of a 1x1 array sits 5 decades below the top one) has no per-layer guarantee
            scale = max(np.abs(ref.Vt).max(), np.abs(ref.Vb).max())
            assert np.abs(vt[v] - ref.Vt).max() <= vtol * scale
            assert np.abs(vb[v] - ref.Vb).max() <= vtol * scale
        np.testing.assert_allclose(io[v], p.g_sense * vb[v][-1], rtol=1e-15)
        assert st[v]["kcl_rel_error"] <= 1e-6
    return st


@pytest.mark.parametrize("prec", [mca.PREC_FP64, mca.PREC_BF16_SPLIT, mca.PREC_BF16,
                                  mca.PREC_MHAT], ids=["fp64", "bf16split", "bf16", "mhat"])
def test_solve_small_config(prec):
    """32x32, log-uniform g, Newton to 1e-10 (seed 0)."""
    _check_solve(mi.config_small(0), prec, 1e-10)


@pytest.mark.parametrize("prec", [mca.PREC_FP64, mca.PREC_BF16_SPLIT], ids=["fp64", "bf16split"])
@pytest.mark.parametrize("m,n", [(1, 1), (1, 17), (5, 1), (33, 47), (130, 70)])
def test_solve_ragged_shapes(m, n, prec):
    cb = mi.make_crossbar(m, n, 11, nvec=3, g_wire_bot=0.5)
    _check_solve(cb, prec, 1e-11)


@pytest.mark.parametrize("prec", [mca.PREC_FP64, mca.PREC_BF16_SPLIT], ids=["fp64", "bf16split"])
def test_solve_bimodal_256(prec):
    """256x256 bimodal conductances, eight seeds (map s with input vector s)."""
    for seed in range(8):
        _check_solve(mi.config_bimodal(seed), prec, 1e-10, ref_tol=1e-13)


@pytest.mark.parametrize("prec", [mca.PREC_MHAT, mca.PREC_JACOBI, mca.PREC_NONE],
                         ids=["mhat", "jacobi", "none"])
def test_restarted_gmres_other_preconditioners(prec):
    """Restarted FGMRES with the paper-literal, Jacobi and no preconditioner reaches the
    requested relative residual of the linear system (true residual checked here)."""
    cb = mi.make_crossbar(24, 20, 12)
    p = cb.params
    N = 24 * 20
    Dr = cb.gmap.ravel().copy()
    J = O.jacobian(p, cb.gmap, np.zeros(N), np.zeros(N))
    rhs = np.random.default_rng(1).standard_normal(2 * N)
    with mca.Solver(_params(p, precision=prec, max_batch=1), cb.gmap) as s:
        dx = torch.empty(1, 2 * N, dtype=torch.float64, device=DEV)
        its, res = s.gmres_solve(_t(Dr[None]), [Dr.mean()], _t(rhs[None]), dx, 1e-8,
                                 max_iters=20000)
        dx = dx.cpu().numpy()[0]
    assert np.linalg.norm(rhs - J @ dx) <= 1.5e-8 * np.linalg.norm(rhs)
    assert its[0] >= 1


def test_selective_reorthogonalisation_long_cycle():
    """A 30-iteration cycle without preconditioning loses orthogonality fast enough that
    the second Gram-Schmidt pass is taken; the GMRES minimum residual still matches the
    oracle's modified Gram-Schmidt GMRES, and the Givens estimate matches the true
    residual (which needs an orthonormal basis)."""
    cb = mi.make_crossbar(24, 20, 12)
    p = cb.params
    N = 24 * 20
    Dr = cb.gmap.ravel().copy()
    J = O.jacobian(p, cb.gmap, np.zeros(N), np.zeros(N))
    rhs = np.random.default_rng(2).standard_normal(2 * N)
    with mca.Solver(_params(p, precision=mca.PREC_NONE, max_batch=1), cb.gmap) as s:
        s.profile(True)
        dx = torch.empty(1, 2 * N, dtype=torch.float64, device=DEV)
        its, res = s.gmres_solve(_t(Dr[None]), [Dr.mean()], _t(rhs[None]), dx, 1e-15)
        prof = s.profile_read()
        s.profile(False)
        dx = dx.cpu().numpy()[0]
    assert its[0] == 30
    assert prof["reorth"]["launches"] > 0
    assert prof["reorth"]["launches"] < prof["update_norm"]["launches"]
    true_res = np.linalg.norm(rhs - J @ dx)
    np.testing.assert_allclose(res[0], true_res, rtol=1e-6)
    x_ref, _, _ = O.gmres_right(lambda v: J @ v, rhs, lambda v: v, restart=30, rtol=1e-15,
                                maxiter=30)
    np.testing.assert_allclose(true_res, np.linalg.norm(rhs - J @ x_ref), rtol=1e-6)


def test_fp32_first_step_apply_matches_fp64_apply():
    """With eta0 >= 1e-4 the first Newton step runs its Jacobian applies in FP32; with a
    tighter eta0 every apply is FP64.  Both must reach the requested KCL residual and the
    same solution (to the stop test's scale), with the same number of Newton steps."""
    cb = mi.make_crossbar(96, 80, 41, nvec=4, g_wire_bot=0.5)
    p = cb.params
    out = {}
    for eta0 in (1e-3, 5e-5):
        with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, newton_rtol=1e-10,
                                eta0=eta0, max_batch=4), cb.gmap) as s:
            out[eta0] = s.solve(cb.vin)
    for v in range(4):
        for eta0 in out:
            st = out[eta0][3][v]
            assert st["status"] == 0 and st["rel_residual"] <= 1e-10, (eta0, st)
        scale = max(np.abs(out[5e-5][0][v]).max(), np.abs(out[5e-5][1][v]).max())
        assert np.abs(out[1e-3][0][v] - out[5e-5][0][v]).max() <= 1e-7 * scale
        assert np.abs(out[1e-3][1][v] - out[5e-5][1][v]).max() <= 1e-7 * scale
        assert out[1e-3][3][v]["newton_iters"] <= out[5e-5][3][v]["newton_iters"] + 1


def test_batch_matches_single_solves():
    cb = mi.make_crossbar(48, 40, 21, nvec=6)
    p = cb.params
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=4,
                            newton_rtol=1e-11), cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=1,
                            newton_rtol=1e-11), cb.gmap) as s:
        for v in range(6):
            vt1, vb1, io1, st1 = s.solve(cb.vin[v:v + 1])
            assert _rel_err(vt[v], vt1[0]) < 1e-9 and _rel_err(vb[v], vb1[0]) < 1e-8


def test_multi_pass_output_pipelining():
    """A call with more vectors than max_batch runs in passes whose output copies overlap
    the next pass (double-buffered state): 10 vectors in passes of 3 (one ragged) must give
    the per-vector results, into host and into device buffers."""
    cb = mi.make_crossbar(40, 36, 31, nvec=10)
    p = cb.params
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=3,
                            newton_rtol=1e-11), cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
        dvt = torch.empty(10, 40, 36, dtype=torch.float64, device=DEV)
        dvb = torch.empty_like(dvt)
        dio = torch.empty(10, 36, dtype=torch.float64, device=DEV)
        s.solve(_t(cb.vin), dvt, dvb, dio)
        singles = [s.solve(cb.vin[v:v + 1]) for v in range(10)]
    for v in range(10):
        assert st[v]["status"] == 0
        assert _rel_err(vt[v], singles[v][0][0]) < 1e-9
        assert _rel_err(vb[v], singles[v][1][0]) < 1e-8
        np.testing.assert_allclose(io[v], singles[v][2][0], rtol=1e-8)
    np.testing.assert_array_equal(dvt.cpu().numpy(), vt)
    np.testing.assert_array_equal(dvb.cpu().numpy(), vb)
    np.testing.assert_array_equal(dio.cpu().numpy(), io)


def test_multi_pass_warm_start_and_fallback():
    """solve_from over several passes (7 vectors, passes of 3): exact solutions as guesses are
    kept (no Newton work), garbage guesses fall back to V = 0, and every vector ends at the
    plain solve's answer."""
    cb = mi.make_crossbar(24, 28, 33, nvec=7)
    p = cb.params
    N = 24 * 28
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=3,
                            newton_rtol=1e-11), cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
        guess = np.concatenate([vt.reshape(7, N), vb.reshape(7, N)], axis=1)
        guess[1::2] = 1e3                                    # every other guess is garbage
        vt2, vb2, io2, st2 = s.solve_from(cb.vin, _t(guess))
    for v in range(7):
        assert st2[v]["status"] == 0
        assert st2[v]["fallback"] == (1 if v % 2 else 0), (v, st2[v])
        if v % 2 == 0:
            assert st2[v]["newton_iters"] == 0, st2[v]
        assert _rel_err(vt2[v], vt[v]) < 1e-9 and _rel_err(vb2[v], vb[v]) < 1e-8


def test_device_buffers_in_and_out():
    cb = mi.make_crossbar(20, 30, 5, nvec=2)
    p = cb.params
    vin = _t(cb.vin)
    vt = torch.empty(2, 20, 30, dtype=torch.float64, device=DEV)
    vb = torch.empty_like(vt)
    io = torch.empty(2, 30, dtype=torch.float64, device=DEV)
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=2), cb.gmap) as s:
        s.solve(vin, vt, vb, io, stream=torch.cuda.current_stream())
        vt_h, vb_h, io_h, _ = s.solve(cb.vin)
    assert _rel_err(vt.cpu().numpy(), vt_h) < 1e-12
    assert _rel_err(io.cpu().numpy(), io_h) < 1e-12


def test_linear_uniform_single_iteration():
    """Linear devices of one conductance: P = J, so one GMRES iteration and one Newton
    step solve the circuit."""
    cb = mi.make_crossbar(24, 36, 6, b=0.0)
    g = np.full((24, 36), 4e-5)
    p = cb.params
    with mca.Solver(_params(p, precision=mca.PREC_FP64, max_batch=1, newton_rtol=1e-11), g) as s:
        vt, vb, io, st = s.solve(cb.vin)
    assert st[0]["newton_iters"] == 1 and st[0]["gmres_iters"] == 1, st
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, max_batch=1,
                            newton_rtol=1e-9), g) as s:
        vt2, vb2, io2, st2 = s.solve(cb.vin)
    assert st2[0]["status"] == 0 and st2[0]["gmres_iters"] <= 4, st2


def test_bounded_wait_gives_up_and_context_survives():
    """A device wait on a barrier that nothing completes gives up after its limit and
    reports MCA_ERR_TIMEOUT; the context stays usable (a solve afterwards succeeds)."""
    cb = mi.make_crossbar(16, 12, 2)
    with mca.Solver(_params(cb.params, max_batch=1), cb.gmap) as s:
        rc = s.lib.mca_wait_selftest(s.h, 20_000_000)      # 20 ms
        assert rc == mca.ERR_TIMEOUT
        vt, vb, io, st = s.solve(cb.vin)
        assert st[0]["status"] == 0


def test_zero_input_and_status_codes():
    cb = mi.make_crossbar(8, 9, 1)
    p = cb.params
    with mca.Solver(_params(p, max_batch=2), cb.gmap) as s:
        vt, vb, io, st = s.solve(np.zeros((1, 8)))
        assert st[0]["status"] == 0 and np.all(vt == 0) and np.all(vb == 0)
        vt, vb, io, st = s.solve(np.full((1, 8), np.nan), allow_not_converged=True)
        assert st[0]["status"] == mca.ERR_NONFINITE
    with mca.Solver(_params(p, max_batch=1, max_newton=1, newton_rtol=1e-14), cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin, allow_not_converged=True)
        assert st[0]["status"] == mca.ERR_NOT_CONVERGED and st[0]["newton_iters"] == 1
        assert np.all(np.isfinite(vt))
    bad = cb.gmap.copy()
    bad[2, 3] = np.nan
    with pytest.raises(mca.MCAError) as e:
        mca.Solver(_params(p), bad)
    assert e.value.code == mca.ERR_NONFINITE
    bad[2, 3] = -1.0
    with pytest.raises(mca.MCAError) as e:
        mca.Solver(_params(p), bad)
    assert e.value.code == mca.ERR_INVALID_ARG


def test_empty_call_and_batch_and_restart_limits():
    """nvec = 0 is a no-op; a full batch of 64 vectors (max_batch's limit) and the restart
    limits GMRES(1) and GMRES(30) all reach the tolerance on the oracle's residual."""
    cb = mi.make_crossbar(24, 40, 13, nvec=64)
    p = cb.params
    with mca.Solver(_params(p, max_batch=64, newton_rtol=1e-9), cb.gmap) as s:
        vt, vb, io, st = s.solve(np.zeros((0, 24)))
        assert vt.shape == (0, 24, 40) and st == []
        vt, vb, io, st = s.solve(cb.vin)
    for v in range(64):
        assert st[v]["status"] == 0
        Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], vt[v].ravel(), vb[v].ravel())
        Yt, _ = O.source_vector(p, cb.vin[v])
        assert np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt) <= 1.01e-9
    for restart in (1, 30):
        for prec in (mca.PREC_FP64, mca.PREC_BF16_SPLIT):
            with mca.Solver(_params(p, max_batch=2, newton_rtol=1e-9, gmres_restart=restart,
                                    precision=prec), cb.gmap) as s:
                vt, vb, io, st = s.solve(cb.vin[:2])
            for v in range(2):
                assert st[v]["status"] == 0, (restart, prec, st[v])
                Ft, Fb = O.residual(p, cb.gmap, cb.vin[v], vt[v].ravel(), vb[v].ravel())
                Yt, _ = O.source_vector(p, cb.vin[v])
                rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
                assert rel <= 1.01e-9, (restart, prec, rel)


def test_large_rectangular_4096x2048_residual():
    """4096 x 2048 (16.8M unknowns, rectangular, the largest case here): BF16-split
    preconditioner to 1e-8; the oracle recomputes the FP64 KCL residual and the balance."""
    cb = mi.make_crossbar(4096, 2048, 7, g_wire_bot=0.5)
    p = cb.params
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, newton_rtol=1e-8, max_batch=1),
                    cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
    assert st[0]["status"] == 0 and st[0]["gmres_iters"] <= 20
    Ft, Fb = O.residual(p, cb.gmap, cb.vin[0], vt[0].ravel(), vb[0].ravel())
    Yt, _ = O.source_vector(p, cb.vin[0])
    rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
    assert rel <= 1e-8 * 1.01
    assert abs(O.kcl_balance(p, cb.vin[0], vt[0], vb[0])) <= 1e-6 * O.outputs(
        p, cb.vin[0], vt[0], vb[0])["i_in"].sum()


def test_full_size_1024_sampled():
    """1024x1024 (2.1M unknowns), log-uniform g, wires 1 S / 0.5 S, BF16 split
    preconditioner, Newton to 1e-8: the oracle recomputes the FP64 residual of the
    returned voltages, and the voltages match the oracle's preconditioned-GMRES solve."""
    cb = mi.config_large(1024, 0)
    p = cb.params
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, newton_rtol=1e-8, max_batch=1),
                    cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
    assert st[0]["status"] == 0
    Ft, Fb = O.residual(p, cb.gmap, cb.vin[0], vt[0].ravel(), vb[0].ravel())
    Yt, _ = O.source_vector(p, cb.vin[0])
    rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
    assert rel <= 1e-8 * 1.01
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, newton_rtol=1e-12, max_batch=1),
                    cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
    ref = O.newton_solve(p, cb.gmap, cb.vin[0], tol=1e-12, linear="pgmres")
    assert _rel_err(vt[0], ref.Vt) <= 1e-7 and _rel_err(vb[0], ref.Vb) <= 1e-7


def test_full_size_2048_residual():
    """2048x2048 (8.4M unknowns), log-uniform g, wires 1 S / 0.5 S, BF16 split
    preconditioner, Newton to 1e-8: the oracle recomputes the FP64 KCL residual of the
    returned voltages and the Kirchhoff balance."""
    cb = mi.config_large(2048, 0)
    p = cb.params
    with mca.Solver(_params(p, precision=mca.PREC_BF16_SPLIT, newton_rtol=1e-8, max_batch=1),
                    cb.gmap) as s:
        vt, vb, io, st = s.solve(cb.vin)
    assert st[0]["status"] == 0 and st[0]["gmres_iters"] <= 20
    Ft, Fb = O.residual(p, cb.gmap, cb.vin[0], vt[0].ravel(), vb[0].ravel())
    Yt, _ = O.source_vector(p, cb.vin[0])
    rel = np.linalg.norm(np.concatenate([Ft, Fb])) / np.linalg.norm(Yt)
    assert rel <= 1e-8 * 1.01
    assert abs(O.kcl_balance(p, cb.vin[0], vt[0], vb[0])) <= 1e-6 * O.outputs(
        p, cb.vin[0], vt[0], vb[0])["i_in"].sum()
