"""CPU FP64 oracle for the steady-state memristor-crossbar (MCA) solve.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  It shares no code with the CUDA
library and never imports it; the seeded inputs come from ``mca_inputs``.

Everything is plain NumPy / SciPy in float64, written in the order and notation of the
paper (Xie et al., "A Fast Method for Steady-State Memristor Crossbar Array Circuit
Simulation", arXiv 2109.07929):

* Section 2, eq. (MNA), eq. (F): the steady-state KCL system
      G_t V_t + I_t(V_t, V_b) - Y_t = 0,   G_b V_b - I_b(V_t, V_b) - Y_b = 0;
* eqs. (Gt), (Gb): G_t = I (x) G (one chain per row), G_b = G (x) I (one chain per
  column), with the natural row-major index i*n + j for both layers (Section 3.1,
  "perpendicular natural indexing");
* eq. (G): the 1-D wire operator, read as a tridiagonal chain Laplacian whose end
  entries carry the terminations (diagonal 2g inside, g + g_end at the ends);
* eq. (Newton3), eq. (J): Newton on F with J = blockdiag(G_t, G_b) + the diagonal
  device blocks;
* eq. (P): the preconditioner with a1 = a2 = mean device conductance (Section 3.1);
* eq. (block), eq. (M): block inversion with the Schur complement
  M = -a2 I + (1/a1) G_2 (x) G_1, G_1 = G_r + a1 I, G_2 = G_c + a2 I;
* eqs. (diagM), (condition), (Mhat), (G2hat), (M-1hat), (2matrix1-4): the paper's
  approximation M ~ M_hat applied as a1 * G_2^-1 X G_1^-1;
* Section 4: GMRES with relative tolerance 1e-6 per linear solve.

The device model is i = (g/b) sinh(b dV) (b = 0 means the linear limit i = g dV);
the paper's Yakopcic parameters are not given.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import scipy.linalg as sla


# ----------------------------------------------------------------------------------
# Circuit operators (Section 2; eqs. G, Gt, Gb, F, J)
# ----------------------------------------------------------------------------------

def wire_diagonal(n, g, g_first, g_last):
    """Diagonal of the 1-D wire operator of eq. (G) for a chain of n nodes with segment
    conductance g, node 0 tied to its source/ground through g_first and node n-1
    through g_last.  Inside nodes see two segments (2g)."""
    d = np.empty(n)
    for j in range(n):
        left = g_first if j == 0 else g
        right = g_last if j == n - 1 else g
        d[j] = left + right
    return d


def wire_matrix(n, g, g_first, g_last):
    """Dense 1-D wire operator of eq. (G): tridiag(-g, d, -g)."""
    d = wire_diagonal(n, g, g_first, g_last)
    G = np.diag(d)
    for j in range(n - 1):
        G[j, j + 1] = -g
        G[j + 1, j] = -g
    return G


def row_operator(p):
    """G_r: one top-layer row (word line), left end via g_src, right end via 1 kohm."""
    return wire_matrix(p.cols, p.g_wire_top, p.g_src, p.g_term_top_right)


def col_operator(p):
    """G_c: one bottom-layer column (bit line), row 0 end via 1 kohm, row m-1 end
    sensed through g_sense."""
    return wire_matrix(p.rows, p.g_wire_bot, p.g_term_bot_top, p.g_sense)


def layer_operators(p):
    """eq. (Gt): G_t = I_m (x) G_r;  eq. (Gb): G_b = G_c (x) I_n (row-major vec)."""
    Gr = sp.csr_matrix(row_operator(p))
    Gc = sp.csr_matrix(col_operator(p))
    Gt = sp.kron(sp.identity(p.rows), Gr, format="csr")
    Gb = sp.kron(Gc, sp.identity(p.cols), format="csr")
    return Gt, Gb


def source_vector(p, vin):
    """Y_t, Y_b of eq. (MNA): Norton injection g_src * V_in[i] at node (i, 0) of the
    top layer; the bottom layer is sensed at virtual ground so Y_b = 0."""
    Yt = np.zeros(p.rows * p.cols)
    Yt[np.arange(p.rows) * p.cols] = p.g_src * np.asarray(vin, dtype=np.float64)
    Yb = np.zeros(p.rows * p.cols)
    return Yt, Yb


def device_current(g, b, dv, neg_ratio=1.0):
    """Memristor current from top to bottom node.  The experiments of Section 4 use the
    Yakopcic model at fixed (programmed) internal states: a sinh of the voltage with one
    amplitude for positive and another for negative bias.  With g the small-signal
    conductance of the programmed state (a1 x b) and neg_ratio = a2 / a1:
    i = (g/b) sinh(b dv) for dv >= 0 and neg_ratio (g/b) sinh(b dv) for dv < 0
    (b = 0: the linear device g dv, scaled the same way)."""
    dv = np.asarray(dv, dtype=np.float64)
    i = g * dv if b == 0.0 else (g / b) * np.sinh(b * dv)
    if neg_ratio != 1.0:
        i = np.where(dv < 0.0, neg_ratio * i, i)
    return i


def device_conductance(g, b, dv, neg_ratio=1.0):
    """di/d(dv): g cosh(b dv), times neg_ratio where dv < 0 (the derivative on the side of
    dv the device is on); the diagonal of the device blocks of eq. (J)."""
    dv = np.asarray(dv, dtype=np.float64)
    d = np.array(np.broadcast_to(g, dv.shape), dtype=np.float64, copy=True) if b == 0.0 \
        else g * np.cosh(b * dv)
    if neg_ratio != 1.0:
        d = np.where(dv < 0.0, neg_ratio * d, d)
    return d


def _neg_ratio(p):
    return getattr(p, "neg_ratio", 1.0)


def residual(p, gmap, vin, Vt, Vb, ops=None):
    """eq. (F): F = blockdiag(G_t, G_b) [V_t; V_b] + [I_t; -I_b] - [Y_t; Y_b].
    V_t, V_b are flat row-major vectors of length m*n.  Returns (F_t, F_b)."""
    Gt, Gb = ops if ops is not None else layer_operators(p)
    Yt, Yb = source_vector(p, vin)
    i = device_current(gmap.ravel(), p.b, Vt - Vb, _neg_ratio(p))
    Ft = Gt @ Vt + i - Yt
    Fb = Gb @ Vb - i - Yb
    return Ft, Fb


def jacobian(p, gmap, Vt, Vb, ops=None):
    """eq. (J): J = [[G_t, 0], [0, G_b]] + [[dI_t/dV_t, dI_t/dV_b], [-dI_b/dV_t,
    -dI_b/dV_b]] = [[G_t + D, -D], [-D, G_b + D]], D = diag(g cosh(b dV))."""
    Gt, Gb = ops if ops is not None else layer_operators(p)
    D = sp.diags(device_conductance(gmap.ravel(), p.b, Vt - Vb, _neg_ratio(p)))
    return sp.bmat([[Gt + D, -D], [-D, Gb + D]], format="csr")


# ----------------------------------------------------------------------------------
# 1-D eigen setup (separability of eqs. Gt/Gb, Section 3.1)
# ----------------------------------------------------------------------------------

def wire_eig(n, g, g_first, g_last):
    """Eigenpairs of the tridiagonal wire operator: G = Q diag(lam) Q^T, lam ascending.
    Uses LAPACK's symmetric tridiagonal solver through SciPy."""
    d = wire_diagonal(n, g, g_first, g_last)
    e = np.full(max(n - 1, 0), -g)
    if n == 1:
        return d.copy(), np.ones((1, 1))
    lam, Q = sla.eigh_tridiagonal(d, e)
    return lam, Q


def eig_setup(p):
    """(mu, Q_r) for G_r and (nu, Q_c) for G_c."""
    mu, Qr = wire_eig(p.cols, p.g_wire_top, p.g_src, p.g_term_top_right)
    nu, Qc = wire_eig(p.rows, p.g_wire_bot, p.g_term_bot_top, p.g_sense)
    return mu, Qr, nu, Qc


# ----------------------------------------------------------------------------------
# Preconditioner (eqs. P, block, M, Mhat, 2matrix1-4)
# ----------------------------------------------------------------------------------

def precond_matrix(p, a1, a2, ops=None):
    """eq. (P): P = [[G_t + a1 I, -a1 I], [-a2 I, G_b + a2 I]] (sparse)."""
    Gt, Gb = ops if ops is not None else layer_operators(p)
    N = p.rows * p.cols
    I = sp.identity(N)
    return sp.bmat([[Gt + a1 * I, -a1 * I], [-a2 * I, Gb + a2 * I]], format="csr")


def precond_scalars(p, gmap, Vt, Vb):
    """a1 = a2 = mean diagonal of the device conductance block (Section 3.1; the sign
    is taken so that both are the positive average device conductance)."""
    a = float(np.mean(device_conductance(gmap.ravel(), p.b, Vt - Vb, _neg_ratio(p))))
    return a, a


def precond_apply_modes(eig, a1, a2, rt, rb, shape):
    """Exact P^-1 r.  In the Kronecker eigenbasis X_hat = Q_c^T X Q_r every mode
    (i', j') of P decouples into the 2x2 block [[mu_j' + a1, -a1], [-a2, nu_i' + a2]]
    (G_t -> mu_j', G_b -> nu_i'), whose inverse is applied mode by mode; this is
    eq. (block) with the exact Schur complement M of eq. (M)."""
    mu, Qr, nu, Qc = eig
    m, n = shape
    Xt = Qc.T @ rt.reshape(m, n) @ Qr
    Xb = Qc.T @ rb.reshape(m, n) @ Qr
    MU = mu[None, :]
    NU = nu[:, None]
    det = MU * NU + MU * a2 + NU * a1        # (mu + a1)(nu + a2) - a1 a2
    Yt = ((NU + a2) * Xt + a1 * Xb) / det
    Yb = (a2 * Xt + (MU + a1) * Xb) / det
    zt = (Qc @ Yt @ Qr.T).ravel()
    zb = (Qc @ Yb @ Qr.T).ravel()
    return zt, zb


def schur_apply_inverse(eig, a1, a2, w, shape):
    """M^-1 w with M = -a2 I + (1/a1) (G_c + a2 I) (x) (G_r + a1 I) (eq. M), through the
    Kronecker eigenbasis."""
    mu, Qr, nu, Qc = eig
    m, n = shape
    W = Qc.T @ w.reshape(m, n) @ Qr
    lamM = -a2 + (nu[:, None] + a2) * (mu[None, :] + a1) / a1
    return (Qc @ (W / lamM) @ Qr.T).ravel()


def precond_apply_block(p, eig, a1, a2, rt, rb, minv=None):
    """P^-1 r evaluated literally through eq. (block) with A = G_t + a1 I, B = -a1 I,
    C = -a2 I, D = G_b + a2 I:
        z_1 = M^-1 (r_2 - D B^-1 r_1),   z_2 = B^-1 (r_1 - A z_1).
    ``minv`` applies M^-1 (default: the exact eigenbasis form)."""
    Gt, Gb = layer_operators(p)
    shape = (p.rows, p.cols)
    if minv is None:
        minv = lambda w: schur_apply_inverse(eig, a1, a2, w, shape)
    Binv = lambda v: -v / a1
    Dmat = lambda v: Gb @ v + a2 * v
    Amat = lambda v: Gt @ v + a1 * v
    z1 = minv(rb - Dmat(Binv(rt)))
    z2 = Binv(rt - Amat(z1))
    return z1, z2


def mhat_apply_inverse(p, a1, a2, w):
    """Paper's approximation (eqs. Mhat, G2hat, M-1hat, 2matrix1-4): drop -a2 I from M,
    M_hat = (G_2 / a1) (x) G_1, so M_hat^-1 w = a1 * G_2^-1 W G_1^-1 with W the
    row-major m x n reshape of w (G_1 = G_r + a1 I, G_2 = G_c + a2 I), each factor
    applied by a tridiagonal solve."""
    m, n = p.rows, p.cols
    W = w.reshape(m, n)
    d1 = wire_diagonal(n, p.g_wire_top, p.g_src, p.g_term_top_right) + a1
    d2 = wire_diagonal(m, p.g_wire_bot, p.g_term_bot_top, p.g_sense) + a2

    def band(d, g):
        k = d.size
        ab = np.zeros((3, k))
        ab[0, 1:] = -g
        ab[1, :] = d
        ab[2, :-1] = -g
        return ab

    T = sla.solve_banded((1, 1), band(d2, p.g_wire_bot), W)          # G_2^-1 W
    U = sla.solve_banded((1, 1), band(d1, p.g_wire_top), T.T).T      # (.) G_1^-1
    return (a1 * U).ravel()


def mhat_condition(p, a1, a2):
    """eqs. (diagM), (condition): diag(M) = -a2 + (2g + a2)(2g + a1)/a1 and the
    approximation is used when 20 a2 < (2g + a2)(2g + a1)/a1.  Evaluated with the
    weaker of the two wires."""
    g = min(p.g_wire_top, p.g_wire_bot)
    rhs = (2 * g + a2) * (2 * g + a1) / a1
    return 20 * a2 < rhs, -a2 + rhs


# ----------------------------------------------------------------------------------
# GMRES with right preconditioning (Section 4: GMRES, rtol 1e-6)
# ----------------------------------------------------------------------------------

def gmres_right(matvec, rhs, precond, x0=None, restart=30, rtol=1e-6, atol=0.0,
                maxiter=10000):
    """Restarted GMRES(restart) with right preconditioning (A M^-1 u = b, x = M^-1 u),
    modified Gram-Schmidt Arnoldi and Givens rotations (Saad, Iterative Methods for
    Sparse Linear Systems, Alg. 6.9 / 9.5).  Stops when ||b - A x|| <= max(rtol*||b||,
    atol).  Returns (x, total iterations, residual history of the estimates)."""
    n = rhs.size
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(rhs)
    target = max(rtol * bnorm, atol)
    history = []
    its = 0
    if bnorm == 0.0:
        return np.zeros(n), 0, [0.0]
    while its < maxiter:
        r = rhs - matvec(x)
        beta = np.linalg.norm(r)
        history.append(beta)
        if beta <= target:
            break
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        gvec = np.zeros(restart + 1)
        gvec[0] = beta
        V[0] = r / beta
        k_done = 0
        for k in range(restart):
            Z[k] = precond(V[k])
            w = matvec(Z[k])
            for j in range(k + 1):                      # modified Gram-Schmidt
                H[j, k] = np.dot(w, V[j])
                w = w - H[j, k] * V[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0:
                V[k + 1] = w / H[k + 1, k]
            for j in range(k):                          # previous rotations
                t = cs[j] * H[j, k] + sn[j] * H[j + 1, k]
                H[j + 1, k] = -sn[j] * H[j, k] + cs[j] * H[j + 1, k]
                H[j, k] = t
            rho = np.hypot(H[k, k], H[k + 1, k])
            cs[k] = H[k, k] / rho
            sn[k] = H[k + 1, k] / rho
            H[k, k] = rho
            H[k + 1, k] = 0.0
            gvec[k + 1] = -sn[k] * gvec[k]
            gvec[k] = cs[k] * gvec[k]
            its += 1
            k_done = k + 1
            history.append(abs(gvec[k + 1]))
            if abs(gvec[k + 1]) <= target or its >= maxiter:
                break
        y = sla.solve_triangular(H[:k_done, :k_done], gvec[:k_done])
        x = x + Z[:k_done].T @ y
        if history[-1] <= target:
            r = rhs - matvec(x)
            if np.linalg.norm(r) <= target * (1 + 1e-6):
                history.append(np.linalg.norm(r))
                break
    return x, its, history


# ----------------------------------------------------------------------------------
# Newton (eq. Newton3) with a direct or a preconditioned-GMRES linear solve
# ----------------------------------------------------------------------------------

def _interleave_perm(m, n):
    """Permutation taking [V_t; V_b] to the cell-interleaved order (t, b) per cell,
    row-major over cells, which makes J banded with bandwidth 2n."""
    N = m * n
    perm = np.empty(2 * N, dtype=np.int64)
    perm[0::2] = np.arange(N)
    perm[1::2] = N + np.arange(N)
    return perm


def banded_solve(J, rhs, m, n):
    """Solve J x = rhs by banded LU on the interleaved ordering (bandwidth 2n)."""
    perm = _interleave_perm(m, n)
    Jp = J[perm][:, perm].tocoo()
    bw = 2 * n
    N2 = 2 * m * n
    ab = np.zeros((2 * bw + 1, N2))
    ab[bw + Jp.row - Jp.col, Jp.col] = Jp.data
    xp = sla.solve_banded((bw, bw), ab, rhs[perm])
    x = np.empty_like(xp)
    x[perm] = xp
    return x


class SolveResult(dict):
    __getattr__ = dict.__getitem__


def newton_solve(p, gmap, vin, tol=1e-10, linear="direct", max_newton=50,
                 restart=30, gmres_rtol=1e-6, precond="exact", V0=None):
    """Newton iteration of eq. (Newton3) from V^0 = 0 (undamped), stopping when the
    relative KCL residual ||F||_2 / ||Y||_2 <= tol.

    linear = "direct"  : sparse LU (SuperLU) of J;
             "banded"  : banded LU of J on the interleaved ordering;
             "pgmres"  : right-preconditioned GMRES(restart) with rtol gmres_rtol
                         (Section 4), tightened to 0.1 * tol * ||Y|| / ||F|| when that is
                         smaller so the outer tolerance is reachable.
    precond = "exact" (P^-1 of eq. P by modes), "mhat" (eq. block with M_hat),
              "jacobi", "none".
    """
    m, n = p.rows, p.cols
    N = m * n
    ops = layer_operators(p)
    Yt, Yb = source_vector(p, vin)
    ynorm = np.linalg.norm(np.concatenate([Yt, Yb]))
    if V0 is None:
        Vt = np.zeros(N)
        Vb = np.zeros(N)
    else:
        Vt, Vb = V0[0].ravel().copy(), V0[1].ravel().copy()
    eig = eig_setup(p) if linear == "pgmres" and precond in ("exact",) else None
    history = []
    gmres_its = []
    status = "max_newton"
    if ynorm == 0.0:
        Vt[:] = 0.0
        Vb[:] = 0.0
        status = "converged"
        max_newton = 0
    for it in range(max_newton + 1):
        Ft, Fb = residual(p, gmap, vin, Vt, Vb, ops)
        F = np.concatenate([Ft, Fb])
        fn = np.linalg.norm(F)
        history.append(fn / ynorm if ynorm > 0 else 0.0)
        if fn <= tol * ynorm:
            status = "converged"
            break
        if it == max_newton:
            break
        J = jacobian(p, gmap, Vt, Vb, ops)
        if linear == "direct":
            d = spla.spsolve(J.tocsc(), -F)
            gmres_its.append(0)
        elif linear == "banded":
            d = banded_solve(J, -F, m, n)
            gmres_its.append(0)
        elif linear == "pgmres":
            a1, a2 = precond_scalars(p, gmap, Vt, Vb)
            if precond == "exact":
                def pc(v):
                    zt, zb = precond_apply_modes(eig, a1, a2, v[:N], v[N:], (m, n))
                    return np.concatenate([zt, zb])
            elif precond == "mhat":
                def pc(v):
                    z1, z2 = precond_apply_block(
                        p, None, a1, a2, v[:N], v[N:],
                        minv=lambda w: mhat_apply_inverse(p, a1, a2, w))
                    return np.concatenate([z1, z2])
            elif precond == "jacobi":
                dj = J.diagonal()
                pc = lambda v: v / dj
            else:
                pc = lambda v: v
            rt = min(gmres_rtol, 0.1 * tol * ynorm / fn)
            d, its, _ = gmres_right(lambda v: J @ v, -F, pc, restart=restart, rtol=rt)
            gmres_its.append(its)
        else:
            raise ValueError(linear)
        Vt = Vt + d[:N]
        Vb = Vb + d[N:]
    return SolveResult(Vt=Vt.reshape(m, n), Vb=Vb.reshape(m, n), rel_residual=history[-1],
                       history=history, newton_iters=len(history) - 1,
                       gmres_iters=gmres_its, status=status)


# ----------------------------------------------------------------------------------
# Outputs and Kirchhoff bookkeeping
# ----------------------------------------------------------------------------------

def outputs(p, vin, Vt, Vb):
    """Sensed column currents I_out[j] = g_sense * V_b[m-1, j], driver currents
    I_in[i] = g_src (V_in[i] - V_t[i, 0]) and the two leak terms through the 1 kohm
    terminations."""
    Vt = Vt.reshape(p.rows, p.cols)
    Vb = Vb.reshape(p.rows, p.cols)
    i_out = p.g_sense * Vb[-1, :]
    i_in = p.g_src * (np.asarray(vin) - Vt[:, 0])
    leak_top = p.g_term_top_right * Vt[:, -1]
    leak_bot = p.g_term_bot_top * Vb[0, :]
    return dict(i_out=i_out, i_in=i_in, leak_top=leak_top, leak_bot=leak_bot)


def kcl_balance(p, vin, Vt, Vb):
    """Injected minus removed current: sum I_in - sum I_out - sum leaks (0 at the
    exact solution, since every device current leaves the top layer and enters the
    bottom one)."""
    o = outputs(p, vin, Vt, Vb)
    return o["i_in"].sum() - o["i_out"].sum() - o["leak_top"].sum() - o["leak_bot"].sum()
