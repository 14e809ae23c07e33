"""Oracle: frame matrix and projected (local) KKT operator of block AMEn.

Test infrastructure only (see the package header).

Sec. 5: for a TT vector with cores X_1 (1, n1, r1), X_2 (r1, n2, r2),
X_3 (r2, n3, 1), the frame matrix of eq. frame is
    F_{!=d}(i1,i2,i3; r_{d-1}, j_d, r_d) = X_{<d}(i_<d, r_{d-1}) delta(i_d, j_d) X_{>d}(r_d, i_>d),
and the local system of eq. KKT_red projects every block of the KKT matrix:
F^T M F, F^T K F, F^T K^T F.

The operator is given in TT-matrix form with ranks (R1, R2):
    A = sum_{a,b} A1[a] (x) A2[a][b] (x) A3[b]   (dense n_d x n_d matrices),
so the projected operator at core d is the sum over rank indices of
Phi_L (x) A_d (x) Phi_R with interfaces Phi built factor by factor (Sec. 5,
"multiplication of tensor trains factor by factor").

Pins: the interface form equals F^T A F built from the explicit frame
matrix on tiny sizes; with orthonormal X_{<d}, X_{>d} the frame has
orthonormal columns (Sec. 5, last paragraph).
"""
from __future__ import annotations

import numpy as np


def frame_matrix(cores, d):
    """Explicit F_{!=d} of eq. frame, shape (n1 n2 n3, r_{d-1} n_d r_d), C order."""
    X1, X2, X3 = cores
    n = (X1.shape[1], X2.shape[1], X3.shape[1])
    if d == 0:
        right = np.einsum("aib,bj->aij", X2, X3[:, :, 0])            # (r1, n2, n3)
        F = np.einsum("xy,rjk->xjkyr", np.eye(n[0]), right)           # (i1,i2,i3; j1, r1)
        return F.reshape(np.prod(n), n[0] * X1.shape[2])
    if d == 1:
        F = np.einsum("ia,jy,bk->ijkayb", X1[0], np.eye(n[1]), X3[:, :, 0])
        return F.reshape(np.prod(n), X1.shape[2] * n[1] * X2.shape[2])
    left = np.einsum("ia,ajb->ijb", X1[0], X2)                        # (n1, n2, r2)
    F = np.einsum("ijb,ky->ijkby", left, np.eye(n[2]))
    return F.reshape(np.prod(n), X2.shape[2] * n[2])


def tt_matrix_dense(op):
    """Dense sum_{a,b} A1[a] (x) A2[a][b] (x) A3[b]."""
    A1, A2, A3 = op
    out = 0.0
    for a in range(len(A1)):
        for b in range(len(A3)):
            out = out + np.kron(A1[a], np.kron(A2[a][b], A3[b]))
    return out


def local_operator_frame(op, cores, d):
    F = frame_matrix(cores, d)
    return F.T @ tt_matrix_dense(op) @ F


def interfaces(op, cores, d):
    """(PhiL, Ad, PhiR) of the projected operator at core d.

    PhiL: (R_{d-1}, r_{d-1}, r_{d-1}); Ad: (R_{d-1}, R_d) nested lists of
    (n_d, n_d); PhiR: (R_d, r_d, r_d).  R_0 = R_3 = 1, r_0 = r_3 = 1.
    """
    A1, A2, A3 = op
    X1, X2, X3 = cores
    R1, R2 = len(A1), len(A3)
    one = np.ones((1, 1, 1))
    if d == 0:
        PhiL = one
        Ad = [[A1[a] for a in range(R1)]]
        # PhiR1[a](r1, r1') = sum X_{>1}(r1, i2 i3) (A2[a][b] (x) A3[b]) X_{>1}(r1', ...)
        PhiR3 = np.stack([X3[:, :, 0] @ A3[b] @ X3[:, :, 0].T for b in range(R2)])
        PhiR = np.stack([
            sum(np.einsum("aib,ij,cjd,bd->ac", X2, A2[a][b], X2, PhiR3[b]) for b in range(R2))
            for a in range(R1)])
        return PhiL, Ad, PhiR
    if d == 1:
        PhiL = np.stack([X1[0].T @ A1[a] @ X1[0] for a in range(R1)])
        PhiR = np.stack([X3[:, :, 0] @ A3[b] @ X3[:, :, 0].T for b in range(R2)])
        return PhiL, A2, PhiR
    PhiL1 = np.stack([X1[0].T @ A1[a] @ X1[0] for a in range(R1)])
    PhiL = np.stack([
        sum(np.einsum("ac,aib,ij,cjd->bd", PhiL1[a], X2, A2[a][b], X2) for a in range(R1))
        for b in range(R2)])
    Ad = [[A3[b]] for b in range(R2)]
    return PhiL, Ad, one


def local_matvec(PhiL, Ad, PhiR, x):
    """y = sum_{a,b} (PhiL[a] (x) Ad[a][b] (x) PhiR[b]) x, x shaped (r0, n, r1)."""
    y = np.zeros_like(x)
    for a in range(PhiL.shape[0]):
        for b in range(PhiR.shape[0]):
            y += np.einsum("ac,ij,bd,cjd->aib", PhiL[a], Ad[a][b], PhiR[b], x)
    return y


def local_operator_interfaces(PhiL, Ad, PhiR):
    out = 0.0
    for a in range(PhiL.shape[0]):
        for b in range(PhiR.shape[0]):
            out = out + np.kron(PhiL[a], np.kron(Ad[a][b], PhiR[b]))
    return out


def local_kkt_frame(opM, opK, beta, cores, d):
    """Projected KKT matrix of eq. KKT_red (tau = 1), dense."""
    F = frame_matrix(cores, d)
    M = F.T @ tt_matrix_dense(opM) @ F
    K = F.T @ tt_matrix_dense(opK) @ F
    Kt = F.T @ tt_matrix_dense(opK).T @ F
    Z = np.zeros_like(M)
    return np.block([[M, Z, Kt], [Z, beta * M, -M], [K, -M, Z]])
