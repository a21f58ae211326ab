"""Model of a multi-right-hand-side (block) Krylov solve of the first Newton step, to
measure what it would save on the statistical-characterisation workload.

At V = 0 every input vector of one crossbar sees the same Jacobian J(0) (D = g, eq. (J)),
so the first Newton systems J(0) d_s = Y_s (s = 1 .. S, eq. (Newton3) with F(0) = -Y) share
their matrix and could be solved as one block.  Block GMRES (right-preconditioned with the
exact P^-1 of eq. (P), block modified Gram-Schmidt, Householder QR of each new block) is
run until every column's residual is below eta0 times its right-hand side's norm, and
compared with S single right-preconditioned GMRES solves to the same tolerance (the
oracle's gmres_right).  Both count preconditioner applies (= Jacobian applies), the work
unit of the tensor-core path.  Test infrastructure: imports the oracle only.
"""
from __future__ import annotations

import numpy as np

from oracle import mca_oracle as O


def first_step_systems(p, gmap, vins):
    """J(0) (sparse), the exact preconditioner of J(0) and the right-hand sides Y_s."""
    N = p.rows * p.cols
    J = O.jacobian(p, gmap, np.zeros(N), np.zeros(N))
    eig = O.eig_setup(p)
    a1, a2 = O.precond_scalars(p, gmap, np.zeros(N), np.zeros(N))

    def pc(v):
        zt, zb = O.precond_apply_modes(eig, a1, a2, v[:N], v[N:], (p.rows, p.cols))
        return np.concatenate([zt, zb])

    B = np.stack([np.concatenate(O.source_vector(p, v)) for v in vins], axis=1)
    return J, pc, B


def single_gmres_applies(J, pc, B, eta):
    """Preconditioner applies of one GMRES(30) solve per column, to eta ||b||."""
    its = []
    for s in range(B.shape[1]):
        _, k, _ = O.gmres_right(lambda x: J @ x, B[:, s], pc, restart=30, rtol=eta)
        its.append(k)
    return its


def block_gmres_applies(J, pc, B, eta, max_blocks=30):
    """Block GMRES from X = 0 on J P^-1 U = B, X = P^-1 U; returns (block iterations,
    preconditioner applies, the largest relative residual over the columns, checked on
    the true residual of the returned X)."""
    n, S = B.shape
    bn = np.linalg.norm(B, axis=0)
    V0, R0 = np.linalg.qr(B)                       # B = V0 R0
    Vs = [V0]
    Zs = []
    Hcols = []                                     # block columns of the Hessenberg
    applies = 0
    for k in range(max_blocks):
        Z = np.stack([pc(Vs[k][:, s]) for s in range(S)], axis=1)
        applies += S
        W = J @ Z
        Zs.append(Z)
        col = []
        for j in range(k + 1):                     # block modified Gram-Schmidt
            Hjk = Vs[j].T @ W
            W = W - Vs[j] @ Hjk
            col.append(Hjk)
        Vn, Hn = np.linalg.qr(W)
        col.append(Hn)
        Vs.append(Vn)
        Hcols.append(col)
        # least squares min || E1 R0 - H Y || over the (k+2) S x (k+1) S block Hessenberg
        H = np.zeros(((k + 2) * S, (k + 1) * S))
        for c, blocks in enumerate(Hcols):
            for r, blk in enumerate(blocks):
                H[r * S:(r + 1) * S, c * S:(c + 1) * S] = blk
        E = np.zeros(((k + 2) * S, S))
        E[:S] = R0
        Y, *_ = np.linalg.lstsq(H, E, rcond=None)
        res = np.linalg.norm(E - H @ Y, axis=0) / bn
        if np.all(res <= eta):
            X = np.concatenate(Zs, axis=1) @ Y
            true = np.linalg.norm(B - J @ X, axis=0) / bn
            return k + 1, applies, float(true.max())
    raise RuntimeError("block GMRES did not converge")
