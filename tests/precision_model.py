"""NumPy model of the tensor-core preconditioner's arithmetic, used to choose which
operands of the four eigenbasis transforms need more than one BF16 word.

The preconditioner z = P^-1 r (eqs. (P), (block), (M); the tensor-product evaluation of
Section 3.2 in the exact Kronecker eigenbasis) is four GEMMs per layer:

    1: T1 = X Q_r            2: Y_hat = modes^-1 (Q_c^T T1)
    3: E  = Y_hat Q_r^T      4: Z     = Q_c E

Every operand is rounded to BF16 (round to nearest even on the float32 bit pattern) and
every product accumulates in float32, as tcgen05 kind::f16 does.  A "split" operand is
carried as hi + lo BF16 words (lo = bf16(x - hi)); a product of two split operands is
hi*hi + hi*lo + lo*hi (the lo*lo term is below FP32 rounding).  The variants:

    fp64         the exact preconditioner (no rounding)
    bf16         every operand one BF16 word
    fp16         every operand one FP16 word (each operand scaled to its own maximum)
    split3       transforms 1, 2 plain; 3 and 4 with both operands split (3 products)
    split2       transform 3 with only Q_r split (Y_hat one word: 2 products), 4 as split3

Newton + right-preconditioned GMRES(30) follow the solver's control: the first linear
solve to a forcing term eta0 = 1e-3, later ones to Eisenstat-Walker 0.9 (|F_k|/|F_k-1|)^2
capped at 1e-2 and never tighter than 0.5 tol |Y| / |F|; the residual, the Jacobian and
the Krylov arithmetic are the oracle's FP64 ones.  The model is test infrastructure: it
imports the oracle and nothing of the CUDA library.
"""
from __future__ import annotations

import numpy as np

from oracle import mca_oracle as O

VARIANTS = ("fp64", "fp16", "bf16", "split3", "split2")


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), returned as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def fp16(x):
    """Round to FP16 after scaling the operand to a maximum of 1 (no overflow)."""
    x = np.asarray(x, dtype=np.float32)
    s = float(np.abs(x).max()) or 1.0
    return (x / s).astype(np.float16).astype(np.float32) * np.float32(s)


def split(x):
    """hi + lo BF16 words of a float32 operand."""
    hi = bf16(x)
    return hi, bf16(np.asarray(x, np.float32) - hi)


def _mm(a, b):
    return np.matmul(a, b, dtype=np.float32)


def _prod(a, b, sa, sb):
    """a @ b with a split into hi + lo when sa, b when sb (FP32 accumulation)."""
    ah, al = split(a) if sa else (bf16(a), None)
    bh, bl = split(b) if sb else (bf16(b), None)
    out = _mm(ah, bh)
    if sa:
        out += _mm(al, bh)
    if sb:
        out += _mm(ah, bl)
    return out


class Precond:
    """P^-1 of one crossbar in a given arithmetic."""

    def __init__(self, p, variant):
        assert variant in VARIANTS, variant
        self.p = p
        self.variant = variant
        self.eig = O.eig_setup(p)
        mu, Qr, nu, Qc = self.eig
        self.mu = mu.astype(np.float32)
        self.nu = nu.astype(np.float32)
        self.Qr = Qr.astype(np.float32)
        self.Qc = Qc.astype(np.float32)

    def __call__(self, a, v):
        p = self.p
        m, n = p.rows, p.cols
        N = m * n
        if self.variant == "fp64":
            zt, zb = O.precond_apply_modes(self.eig, a, a, v[:N], v[N:], (m, n))
            return np.concatenate([zt, zb])
        rnd = fp16 if self.variant == "fp16" else bf16
        X = np.stack([v[:N].reshape(m, n), v[N:].reshape(m, n)]).astype(np.float32)
        Qr, Qc = self.Qr, self.Qc
        T1 = rnd(_mm(rnd(X), rnd(Qr)))                      # transform 1, one-word output
        Xh = _mm(rnd(Qc.T)[None], T1)                       # transform 2
        af = np.float32(a)
        MU = self.mu[None, :]
        NU = self.nu[:, None]
        det = (MU + af) * (NU + af) - af * af               # the FP32 modes epilogue
        Yt = ((NU + af) * Xh[0] + af * Xh[1]) / det
        Yb = (af * Xh[0] + (MU + af) * Xh[1]) / det
        Y = np.stack([Yt, Yb]).astype(np.float32)
        if self.variant in ("bf16", "fp16"):
            E = rnd(_mm(rnd(Y), rnd(Qr.T)))
            Z = _mm(rnd(Qc)[None], E)
        else:
            s3 = self.variant == "split3"
            E = _prod(Y, Qr.T, s3, True)                    # transform 3
            Z = np.stack([_prod(Qc, E[l], True, True) for l in range(2)])   # transform 4
        return np.concatenate([Z[0].ravel(), Z[1].ravel()]).astype(np.float64)


def newton_gmres(p, gmap, vin, variant, tol=1e-8, eta0=1e-3, eta_max=1e-2, restart=30):
    """Newton with right-preconditioned GMRES(restart) under the solver's forcing terms;
    returns (newton steps, GMRES iterations per step, final ||F||/||Y||)."""
    m, n = p.rows, p.cols
    N = m * n
    ops = O.layer_operators(p)
    Yt, Yb = O.source_vector(p, vin)
    ynorm = np.linalg.norm(np.concatenate([Yt, Yb]))
    pc = Precond(p, variant)
    Vt = np.zeros(N)
    Vb = np.zeros(N)
    its = []
    fprev = None
    while True:
        Ft, Fb = O.residual(p, gmap, vin, Vt, Vb, ops)
        F = np.concatenate([Ft, Fb])
        fn = np.linalg.norm(F)
        if fn <= tol * ynorm or len(its) >= 10:
            return len(its), its, fn / ynorm
        eta = eta0 if fprev is None else min(eta_max, 0.9 * (fn / fprev) ** 2)
        eta = min(max(eta, 0.5 * tol * ynorm / fn), 0.5)
        fprev = fn
        J = O.jacobian(p, gmap, Vt, Vb, ops)
        a, _ = O.precond_scalars(p, gmap, Vt, Vb)
        d, k, _ = O.gmres_right(lambda x: J @ x, -F, lambda x: pc(a, x), restart=restart,
                                rtol=eta, maxiter=300)
        its.append(k)
        Vt = Vt + d[:N]
        Vb = Vb + d[N:]
