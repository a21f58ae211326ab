"""Pins for the CPU oracle: each test checks the oracle against something other than
itself (an independent netlist assembly, brute force, a closed form, an invariant of the
circuit or of the algebra, a library routine, or the trend of the paper's Table 1)."""
import json
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import mca_inputs as mi
from oracle import mca_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(m, n, **kw):
    base = dict(g_wire_top=1.0, g_wire_bot=0.5, g_src=0.1, g_term_top_right=1e-3,
                g_term_bot_top=2e-3, g_sense=0.2, b=2.0)
    base.update(kw)
    return mi.CrossbarParams(rows=m, cols=n, **base)


def _netlist_residual(p, gmap, vin, Vt, Vb):
    """KCL at every node written from the circuit: walk over every resistor and every
    memristor and add the current leaving each node (independent of the Kronecker form)."""
    m, n = p.rows, p.cols
    Ft = np.zeros((m, n))
    Fb = np.zeros((m, n))
    Vt = Vt.reshape(m, n)
    Vb = Vb.reshape(m, n)
    for i in range(m):
        for j in range(n - 1):                       # top wire segments along a row
            cur = p.g_wire_top * (Vt[i, j] - Vt[i, j + 1])
            Ft[i, j] += cur
            Ft[i, j + 1] -= cur
        Ft[i, 0] += p.g_src * (Vt[i, 0] - vin[i])    # driver through 10 ohm
        Ft[i, n - 1] += p.g_term_top_right * Vt[i, n - 1]
    for j in range(n):
        for i in range(m - 1):                       # bottom wire segments along a column
            cur = p.g_wire_bot * (Vb[i, j] - Vb[i + 1, j])
            Fb[i, j] += cur
            Fb[i + 1, j] -= cur
        Fb[0, j] += p.g_term_bot_top * Vb[0, j]
        Fb[m - 1, j] += p.g_sense * Vb[m - 1, j]
    for i in range(m):
        for j in range(n):
            dv = Vt[i, j] - Vb[i, j]
            if p.b == 0:
                cur = gmap[i, j] * dv
            else:
                cur = gmap[i, j] / p.b * np.sinh(p.b * dv)
            if dv < 0:                                  # Yakopcic form: a2/a1 below zero
                cur *= p.neg_ratio
            Ft[i, j] += cur
            Fb[i, j] -= cur
    return Ft.ravel(), Fb.ravel()


SHAPES = [(1, 1), (1, 4), (3, 1), (2, 3), (4, 5), (5, 4), (6, 6)]


@pytest.mark.parametrize("m,n", SHAPES)
def test_residual_matches_netlist(m, n):
    rng = np.random.default_rng(7 + m * 10 + n)
    p = _params(m, n)
    g = 10 ** rng.uniform(-6, -3, size=(m, n))
    vin = rng.uniform(0, 0.3, size=m)
    Vt = rng.uniform(-0.2, 0.4, size=m * n)
    Vb = rng.uniform(-0.2, 0.2, size=m * n)
    Ft, Fb = O.residual(p, g, vin, Vt, Vb)
    Rt, Rb = _netlist_residual(p, g, vin, Vt, Vb)
    np.testing.assert_allclose(Ft, Rt, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Fb, Rb, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("m,n", [(3, 4), (5, 2)])
def test_jacobian_finite_difference(m, n):
    rng = np.random.default_rng(3)
    p = _params(m, n, b=3.0)
    g = 10 ** rng.uniform(-4, -2, size=(m, n))
    vin = rng.uniform(0, 0.3, size=m)
    Vt = rng.uniform(-0.3, 0.5, size=m * n)
    Vb = rng.uniform(-0.3, 0.3, size=m * n)
    J = O.jacobian(p, g, Vt, Vb).toarray()
    N = m * n
    h = 1e-6
    Jfd = np.zeros_like(J)
    x = np.concatenate([Vt, Vb])
    for k in range(2 * N):
        xp = x.copy(); xp[k] += h
        xm = x.copy(); xm[k] -= h
        Fp = np.concatenate(O.residual(p, g, vin, xp[:N], xp[N:]))
        Fm = np.concatenate(O.residual(p, g, vin, xm[:N], xm[N:]))
        Jfd[:, k] = (Fp - Fm) / (2 * h)
    np.testing.assert_allclose(J, Jfd, rtol=1e-7, atol=1e-10)


def test_jacobian_is_spd():
    rng = np.random.default_rng(11)
    p = _params(4, 6)
    g = 10 ** rng.uniform(-6, -4, size=(4, 6))
    Vt = rng.uniform(-0.5, 0.5, size=24)
    Vb = rng.uniform(-0.5, 0.5, size=24)
    J = O.jacobian(p, g, Vt, Vb).toarray()
    np.testing.assert_allclose(J, J.T, atol=0)
    assert np.linalg.eigvalsh(J).min() > 0


def test_one_by_one_crossbar_bisection():
    """m = n = 1: eliminate V_b = i(u) / (g_T + g_S) and V_t = u + V_b; the top KCL is a
    strictly increasing scalar function of u = V_t - V_b, solved by bisection."""
    p = _params(1, 1, b=2.0, g_src=0.1, g_term_top_right=1e-3, g_term_bot_top=1e-3,
                g_sense=0.1)
    g = np.array([[3e-2]])
    vin = np.array([0.7])
    gt_end = p.g_src + p.g_term_top_right
    gb_end = p.g_term_bot_top + p.g_sense

    def f(u):
        i = g[0, 0] / p.b * np.sinh(p.b * u)
        return gt_end * (u + i / gb_end) + i - p.g_src * vin[0]

    lo, hi = -1.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    u = 0.5 * (lo + hi)
    vb = g[0, 0] / p.b * np.sinh(p.b * u) / gb_end
    vt = u + vb
    r = O.newton_solve(p, g, vin, tol=1e-14, linear="direct")
    assert r.status == "converged"
    np.testing.assert_allclose(r.Vt[0, 0], vt, rtol=1e-12)
    np.testing.assert_allclose(r.Vb[0, 0], vb, rtol=1e-11)


def _dense_newton(p, g, vin, tol):
    """Newton with numpy.linalg.solve on the dense netlist Jacobian (finite differences of
    the netlist residual are not needed: the netlist KCL is differentiated by hand)."""
    m, n = p.rows, p.cols
    N = m * n
    x = np.zeros(2 * N)
    Ynorm = p.g_src * np.linalg.norm(vin)
    for _ in range(60):
        Ft, Fb = _netlist_residual(p, g, vin, x[:N], x[N:])
        F = np.concatenate([Ft, Fb])
        if np.linalg.norm(F) <= tol * Ynorm:
            break
        J = np.zeros((2 * N, 2 * N))
        h = 1e-7
        for k in range(2 * N):                       # column by column, central
            xp = x.copy(); xp[k] += h
            xm = x.copy(); xm[k] -= h
            J[:, k] = (np.concatenate(_netlist_residual(p, g, vin, xp[:N], xp[N:]))
                       - np.concatenate(_netlist_residual(p, g, vin, xm[:N], xm[N:]))) / (2 * h)
        x = x - np.linalg.solve(J, F)
    return x[:N].reshape(m, n), x[N:].reshape(m, n)


@pytest.mark.parametrize("m,n", [(2, 3), (4, 4), (3, 5)])
def test_newton_matches_dense_bruteforce(m, n):
    rng = np.random.default_rng(5)
    p = _params(m, n)
    g = 10 ** rng.uniform(-4, -2, size=(m, n))
    vin = rng.uniform(0, 0.3, size=m)
    Vt_ref, Vb_ref = _dense_newton(p, g, vin, 1e-13)
    for lin in ("direct", "banded", "pgmres"):
        r = O.newton_solve(p, g, vin, tol=1e-13, linear=lin)
        assert r.status == "converged", lin
        np.testing.assert_allclose(r.Vt, Vt_ref, rtol=1e-7, atol=1e-12)
        np.testing.assert_allclose(r.Vb, Vb_ref, rtol=1e-7, atol=1e-12)


def test_linear_uniform_preconditioner_is_exact():
    """Linear devices of one conductance: D = g0 I = a1 I = a2 I, so P = J and right-
    preconditioned GMRES converges in one iteration, Newton in one step."""
    p = _params(12, 9, b=0.0)
    g = np.full((12, 9), 3e-5)
    vin = np.random.default_rng(2).uniform(0, 0.3, size=12)
    r = O.newton_solve(p, g, vin, tol=1e-11, linear="pgmres")
    assert r.status == "converged"
    assert r.newton_iters == 1
    assert r.gmres_iters == [1]


def test_dst_closed_form_eigenpairs():
    """With both ends tied through g (the paper's eq. G), the wire operator is
    tridiag(-g, 2g, -g): lam_k = 2g - 2g cos(k pi / (n+1)), q_jk = sqrt(2/(n+1))
    sin(j k pi / (n+1))  (DST-I)."""
    n, g = 17, 0.7
    lam, Q = O.wire_eig(n, g, g, g)
    k = np.arange(1, n + 1)
    lam_ref = 2 * g - 2 * g * np.cos(k * np.pi / (n + 1))
    np.testing.assert_allclose(lam, lam_ref, rtol=1e-13, atol=1e-14)
    j = np.arange(1, n + 1)[:, None]
    Qref = np.sqrt(2.0 / (n + 1)) * np.sin(j * k[None, :] * np.pi / (n + 1))
    sign = np.sign(np.sum(Q * Qref, axis=0))
    np.testing.assert_allclose(Q * sign[None, :], Qref, atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 7, 64])
def test_eig_general_ends(n):
    g, g0, g1 = 1.0, 0.1, 1e-3
    lam, Q = O.wire_eig(n, g, g0, g1)
    G = O.wire_matrix(n, g, g0, g1)
    np.testing.assert_allclose(G @ Q, Q * lam[None, :], atol=1e-13)
    np.testing.assert_allclose(Q.T @ Q, np.eye(n), atol=1e-13)
    assert np.all(np.diff(lam) > 0)


@pytest.mark.parametrize("m,n", [(3, 4), (5, 5), (6, 2)])
def test_preconditioner_block_inverse(m, n):
    """Per-mode 2x2 inverse == eq. (block) with the exact Schur complement of eq. (M) ==
    the dense inverse of eq. (P)."""
    rng = np.random.default_rng(9)
    p = _params(m, n)
    eig = O.eig_setup(p)
    a1 = a2 = 3e-2
    P = O.precond_matrix(p, a1, a2).toarray()
    r = rng.standard_normal(2 * m * n)
    z_ref = np.linalg.solve(P, r)
    zt, zb = O.precond_apply_modes(eig, a1, a2, r[:m * n], r[m * n:], (m, n))
    np.testing.assert_allclose(np.concatenate([zt, zb]), z_ref, rtol=1e-10, atol=1e-12)
    z1, z2 = O.precond_apply_block(p, eig, a1, a2, r[:m * n], r[m * n:])
    np.testing.assert_allclose(np.concatenate([z1, z2]), z_ref, rtol=1e-8, atol=1e-10)
    # unequal a1, a2 exercise the separate slots of eq. (P)
    P2 = O.precond_matrix(p, 2e-2, 5e-2).toarray()
    zt, zb = O.precond_apply_modes(eig, 2e-2, 5e-2, r[:m * n], r[m * n:], (m, n))
    np.testing.assert_allclose(np.concatenate([zt, zb]), np.linalg.solve(P2, r),
                               rtol=1e-10, atol=1e-12)


def test_schur_complement_dense():
    """eq. (M): M = C - D B^-1 A equals -a2 I + (1/a1) (G_c + a2 I) (x) (G_r + a1 I)."""
    p = _params(3, 4)
    a1, a2 = 2e-2, 3e-2
    Gt, Gb = O.layer_operators(p)
    N = 12
    I = np.eye(N)
    A = Gt.toarray() + a1 * I
    B = -a1 * I
    C = -a2 * I
    D = Gb.toarray() + a2 * I
    M = C - D @ np.linalg.inv(B) @ A
    G1 = O.row_operator(p) + a1 * np.eye(4)
    G2 = O.col_operator(p) + a2 * np.eye(3)
    np.testing.assert_allclose(M, -a2 * I + np.kron(G2, G1) / a1, rtol=1e-12, atol=1e-12)
    w = np.random.default_rng(1).standard_normal(N)
    np.testing.assert_allclose(O.schur_apply_inverse(O.eig_setup(p), a1, a2, w, (3, 4)),
                               np.linalg.solve(M, w), rtol=1e-9)


def test_mhat_apply_and_condition():
    """eqs. (Mhat), (M-1hat), (2matrix4): M_hat^-1 w = a1 (G_2^-1 (x) G_1^-1) w; and the
    condition of eq. (condition) holds in the operating regime (a ~ 1e-5 << g)."""
    p = _params(4, 5)
    a1, a2 = 2e-5, 2e-5
    G1 = O.row_operator(p) + a1 * np.eye(5)
    G2 = O.col_operator(p) + a2 * np.eye(4)
    w = np.random.default_rng(4).standard_normal(20)
    ref = a1 * np.kron(np.linalg.inv(G2), np.linalg.inv(G1)) @ w
    np.testing.assert_allclose(O.mhat_apply_inverse(p, a1, a2, w), ref, rtol=1e-10)
    ok, diagM = O.mhat_condition(p, a1, a2)
    assert ok and diagM > 20 * a2


def _dense_schur(p, a1, a2):
    """eq. (M) formed densely as the Schur complement C - D B^-1 A of P (eq. P)."""
    Gt, Gb = O.layer_operators(p)
    N = p.rows * p.cols
    I = np.eye(N)
    return -a2 * I - (Gb.toarray() + a2 * I) @ np.linalg.inv(-a1 * I) @ (Gt.toarray() + a1 * I)


@pytest.mark.parametrize("a", [2e-5, 0.3, 0.5, 1.0, 3.0])
def test_mhat_condition_against_dense_schur_diagonal(a):
    """eqs. (diagM), (condition): diag(M) at an interior node is read off the dense
    Schur complement, and the condition 20 a2 < diag(M) + a2 is decided on it.  With
    equal wires the function's diag(M) is that entry; with unequal wires it is the entry
    of the array whose wires are both the weaker one, which bounds every interior entry of
    the actual M from below.  The a values straddle the point where the condition fails."""
    m, n = 5, 6
    interior = [i * n + j for i in range(1, m - 1) for j in range(1, n - 1)]
    for gt, gb in ((1.0, 1.0), (1.0, 0.5), (0.4, 2.0)):
        p = _params(m, n, g_wire_top=gt, g_wire_bot=gb)
        ok, diagM = O.mhat_condition(p, a, a)
        gw = min(gt, gb)
        M_weak = _dense_schur(_params(m, n, g_wire_top=gw, g_wire_bot=gw), a, a)
        d_weak = np.diag(M_weak)[interior]
        np.testing.assert_allclose(d_weak, diagM, rtol=1e-12)
        assert ok == bool(20 * a < d_weak[0] + a)
        d_true = np.diag(_dense_schur(p, a, a))[interior]
        assert diagM <= d_true.min() * (1 + 1e-12)
        if gt == gb:
            np.testing.assert_allclose(d_true, diagM, rtol=1e-12)


def test_kcl_conservation_and_outputs():
    cb = mi.config_small(0)
    p = cb.params
    r = O.newton_solve(p, cb.gmap, cb.vin[0], tol=1e-12, linear="direct")
    o = O.outputs(p, cb.vin[0], r.Vt, r.Vb)
    injected = o["i_in"].sum()
    bal = O.kcl_balance(p, cb.vin[0], r.Vt, r.Vb)
    assert abs(bal) <= 1e-10 * abs(injected)
    # sensed currents are positive and below the injected total
    assert np.all(o["i_out"] > 0) and o["i_out"].sum() < injected


def test_superposition_linear_devices():
    p = _params(5, 7, b=0.0)
    rng = np.random.default_rng(8)
    g = 10 ** rng.uniform(-6, -4, size=(5, 7))
    v1, v2 = rng.uniform(0, 0.3, size=(2, 5))
    s1 = O.newton_solve(p, g, v1, tol=1e-13)
    s2 = O.newton_solve(p, g, v2, tol=1e-13)
    s3 = O.newton_solve(p, g, 2.0 * v1 - 0.5 * v2, tol=1e-13)
    np.testing.assert_allclose(s3.Vt, 2.0 * s1.Vt - 0.5 * s2.Vt, rtol=1e-9, atol=1e-14)
    np.testing.assert_allclose(s3.Vb, 2.0 * s1.Vb - 0.5 * s2.Vb, rtol=1e-9, atol=1e-14)


def test_zero_input_gives_zero():
    cb = mi.make_crossbar(6, 5, 3)
    r = O.newton_solve(cb.params, cb.gmap, np.zeros(6), tol=1e-10)
    assert r.status == "converged"
    assert np.all(r.Vt == 0) and np.all(r.Vb == 0)


def test_gmres_matches_scipy_and_true_residual():
    cb = mi.make_crossbar(8, 9, 12)
    p = cb.params
    N = 72
    Vt = np.zeros(N); Vb = np.zeros(N)
    J = O.jacobian(p, cb.gmap, Vt, Vb)
    rhs = np.random.default_rng(0).standard_normal(2 * N)
    x, its, hist = O.gmres_right(lambda v: J @ v, rhs, lambda v: v, restart=10, rtol=1e-10)
    true_res = np.linalg.norm(rhs - J @ x)
    assert true_res <= 1e-10 * np.linalg.norm(rhs) * 1.01
    x_ref = spla.spsolve(J.tocsc(), rhs)
    np.testing.assert_allclose(x, x_ref, rtol=1e-6, atol=1e-9 * np.abs(x_ref).max())
    # the Givens residual estimate of the last cycle equals the true residual
    xs, _, hs = O.gmres_right(lambda v: J @ v, rhs, lambda v: v, restart=200, rtol=1e-8)
    np.testing.assert_allclose(hs[-1], np.linalg.norm(rhs - J @ xs), rtol=1e-4)


def test_paper_regime_iteration_trend():
    """Table 1 trend: with the proposed preconditioner the GMRES step count stays nearly
    flat with the crossbar size, while unpreconditioned GMRES grows steeply.  (Exact
    counts are not reproducible: the device parameters are not given.)"""
    with open(os.path.join(GOLDEN, "table1_iterations.json")) as f:
        t1 = json.load(f)
    sizes = [16, 32, 64]
    steps_none, steps_prop = [], []
    for n in sizes:
        cb = mi.config_paper_regime(n, 0)
        p = cb.params
        N = n * n
        Vz = np.zeros(N)
        J = O.jacobian(p, cb.gmap, Vz, Vz)
        Yt, Yb = O.source_vector(p, cb.vin[0])
        rhs = np.concatenate([Yt, Yb])
        a1, a2 = O.precond_scalars(p, cb.gmap, Vz, Vz)
        eig = O.eig_setup(p)
        pc = lambda v: np.concatenate(O.precond_apply_modes(eig, a1, a2, v[:N], v[N:], (n, n)))
        _, it_p, _ = O.gmres_right(lambda v: J @ v, rhs, pc, restart=200, rtol=1e-6)
        _, it_n, _ = O.gmres_right(lambda v: J @ v, rhs, lambda v: v, restart=2000, rtol=1e-6)
        steps_prop.append(it_p)
        steps_none.append(it_n)
    paper_prop = t1["steps"]["proposed"][:3]
    paper_none = t1["steps"]["none"][:3]
    # same shape as the paper: flat (within x2 of the paper's counts) vs growing
    assert max(steps_prop) <= 2 * max(paper_prop)
    assert steps_none[-1] >= 3 * steps_none[0]
    assert paper_none[-1] >= 3 * paper_none[0]
    assert all(sn > sp for sn, sp in zip(steps_none, steps_prop))


# ---- planted mistakes: each pin must catch a plausible error in the oracle ---------

def test_pin_catches_transposed_kronecker(monkeypatch):
    """Swapping the Kronecker factors of eqs. (Gt)/(Gb) (top chains along columns,
    bottom along rows) must fail the netlist pin."""
    import scipy.sparse as sp
    p = _params(4, 4)
    rng = np.random.default_rng(1)
    g = 10 ** rng.uniform(-4, -2, size=(4, 4))
    vin = rng.uniform(0, 0.3, size=4)
    Vt = rng.uniform(0, 0.3, size=16)
    Vb = rng.uniform(0, 0.1, size=16)

    def wrong_ops(pp):
        Gr = sp.csr_matrix(O.row_operator(pp))
        Gc = sp.csr_matrix(O.col_operator(pp))
        return (sp.kron(Gr, sp.identity(pp.rows), format="csr"),
                sp.kron(sp.identity(pp.cols), Gc, format="csr"))

    monkeypatch.setattr(O, "layer_operators", wrong_ops)
    Ft, Fb = O.residual(p, g, vin, Vt, Vb)
    Rt, Rb = _netlist_residual(p, g, vin, Vt, Vb)
    assert not (np.allclose(Ft, Rt) and np.allclose(Fb, Rb))


def test_pin_catches_wrong_precond_sign():
    p = _params(3, 4)
    eig = O.eig_setup(p)
    a = 3e-2
    r = np.random.default_rng(2).standard_normal(24)
    z_ref = np.linalg.solve(O.precond_matrix(p, a, a).toarray(), r)
    # the literal sign reading of a1 (mean of dI_t/dV_b < 0) gives a different operator
    zt, zb = O.precond_apply_modes(eig, -a, -a, r[:12], r[12:], (3, 4))
    assert not np.allclose(np.concatenate([zt, zb]), z_ref, rtol=1e-6)


# ---- Yakopcic-form device (asymmetric sinh, Section 4's device model) -------------------

@pytest.mark.parametrize("m,n", [(1, 1), (2, 3), (4, 5), (6, 6)])
@pytest.mark.parametrize("b", [0.0, 2.0])
def test_asymmetric_device_residual_matches_netlist(m, n, b):
    rng = np.random.default_rng(17 + m * 10 + n)
    p = _params(m, n, b=b, neg_ratio=0.35)
    g = 10 ** rng.uniform(-6, -3, size=(m, n))
    vin = rng.uniform(-0.3, 0.3, size=m)
    Vt = rng.uniform(-0.3, 0.3, size=m * n)
    Vb = rng.uniform(-0.2, 0.2, size=m * n)
    Ft, Fb = O.residual(p, g, vin, Vt, Vb)
    Rt, Rb = _netlist_residual(p, g, vin, Vt, Vb)
    np.testing.assert_allclose(Ft, Rt, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(Fb, Rb, rtol=1e-12, atol=1e-15)


def test_asymmetric_device_unit_ratio_is_the_sinh_device():
    rng = np.random.default_rng(2)
    g = 10 ** rng.uniform(-6, -4, size=50)
    dv = rng.uniform(-0.5, 0.5, size=50)
    np.testing.assert_array_equal(O.device_current(g, 2.0, dv, 1.0), g / 2.0 * np.sinh(2.0 * dv))
    np.testing.assert_array_equal(O.device_conductance(g, 2.0, dv, 1.0), g * np.cosh(2.0 * dv))


def test_asymmetric_device_jacobian_finite_difference():
    """Away from dV = 0 (where the model has a kink when a2 != a1) J is the derivative."""
    rng = np.random.default_rng(23)
    m, n = 3, 4
    p = _params(m, n, b=3.0, neg_ratio=0.4)
    N = m * n
    g = 10 ** rng.uniform(-4, -2, size=(m, n))
    vin = rng.uniform(-0.3, 0.3, size=m)
    Vb = rng.uniform(-0.2, 0.2, size=N)
    dv = rng.uniform(0.01, 0.4, size=N) * rng.choice([-1.0, 1.0], size=N)
    Vt = Vb + dv
    J = O.jacobian(p, g, Vt, Vb).toarray()
    h = 1e-6
    Jfd = np.zeros_like(J)
    x = np.concatenate([Vt, Vb])
    for k in range(2 * N):
        xp = x.copy(); xp[k] += h
        xm = x.copy(); xm[k] -= h
        Jfd[:, k] = (np.concatenate(O.residual(p, g, vin, xp[:N], xp[N:]))
                     - np.concatenate(O.residual(p, g, vin, xm[:N], xm[N:]))) / (2 * h)
    np.testing.assert_allclose(J, Jfd, rtol=1e-7, atol=1e-10)
    assert (dv < 0).any() and (dv > 0).any()


@pytest.mark.parametrize("vin0", [0.7, -0.7])
def test_asymmetric_device_one_by_one_bisection(vin0):
    """1x1 array under positive and negative drive: the scalar reduction of the bisection
    pin with the Yakopcic-form current (a2/a1 = 0.3 on the negative side)."""
    r_neg = 0.3
    p = _params(1, 1, b=2.0, neg_ratio=r_neg)
    g = np.array([[3e-2]])
    vin = np.array([vin0])
    gt_end = p.g_src + p.g_term_top_right
    gb_end = p.g_term_bot_top + p.g_sense

    def cur(u):
        i = g[0, 0] / p.b * np.sinh(p.b * u)
        return r_neg * i if u < 0 else i

    def f(u):
        return gt_end * (u + cur(u) / gb_end) + cur(u) - p.g_src * vin[0]

    lo, hi = -1.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
    u = 0.5 * (lo + hi)
    vb = cur(u) / gb_end
    r = O.newton_solve(p, g, vin, tol=1e-14, linear="direct")
    assert r.status == "converged"
    np.testing.assert_allclose(r.Vt[0, 0], u + vb, rtol=1e-12)
    np.testing.assert_allclose(r.Vb[0, 0], vb, rtol=1e-11)
    assert (u < 0) == (vin0 < 0)


def test_asymmetric_device_newton_matches_dense_bruteforce():
    rng = np.random.default_rng(29)
    m, n = 3, 4
    p = _params(m, n, neg_ratio=0.5)
    g = 10 ** rng.uniform(-4, -2, size=(m, n))
    vin = rng.uniform(-0.3, 0.3, size=m)
    Vt_ref, Vb_ref = _dense_newton(p, g, vin, 1e-13)
    for lin in ("direct", "pgmres"):
        r = O.newton_solve(p, g, vin, tol=1e-13, linear=lin)
        assert r.status == "converged", lin
        np.testing.assert_allclose(r.Vt, Vt_ref, rtol=1e-7, atol=1e-12)
        np.testing.assert_allclose(r.Vb, Vb_ref, rtol=1e-7, atol=1e-12)
