"""Oracle: stationary KKT system of the Poisson-constrained control problem.

Test infrastructure only (see the package header).

Sec. 4, eq. KKTSystem, read with one time step (N_t = 1, tau = 1, the
time-difference term dropped) and the desired state entering through the
load vector b (b_i = int yhat beta_i omega):

    [ M    0     K^T ] [y  ]   [b]
    [ 0   beta M  -M ] [u  ] = [0]
    [ K   -M     0   ] [lam]   [0]

Row 1 gives K^T lam = b - M y, row 2 lam = beta u at the optimum, row 3 is
the discrete state equation K y = M u.  Discrete objective
J(y, u) = 1/2 y^T M y - b^T y + 1/2 c + beta/2 u^T M u  (c = int yhat^2 omega),
and along the state equation the reduced gradient is beta M u - M lam with
lam the adjoint K^T lam = b - M y.

For grids too large for the direct solve, `reduced_solve` runs conjugate
gradients on the reduced system (M + beta K M^{-1} K) y = b obtained by
eliminating u and lam (rows 2 and 3), optionally preconditioned by the
Kronecker approximation `kron_schur_preconditioner`.

Pins: the unit-cube fast-diagonalisation solve (independent of SuperLU),
the gradient against central finite differences, first-order optimality of
the KKT solution, and the reduced CG solve against the direct solve on
small curved grids (tests/test_oracle_kkt.py).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def kkt_matrix(M, K, beta):
    Z = None
    return sp.bmat([[M, Z, K.T], [Z, beta * M, -M], [K, -M, Z]], format="csc")


def kkt_rhs(b):
    N = len(b)
    return np.concatenate([b, np.zeros(N), np.zeros(N)])


def kkt_solve(M, K, beta, b):
    """Sparse direct solve (SuperLU) of the stationary KKT system."""
    A = kkt_matrix(M, K, beta)
    z = spla.spsolve(A, kkt_rhs(b))
    N = len(b)
    return z[:N], z[N:2 * N], z[2 * N:]


def kkt_residual(M, K, beta, b, y, u, lam):
    """||rhs - A z||_2 / ||rhs||_2."""
    A = kkt_matrix(M, K, beta)
    r = kkt_rhs(b) - A @ np.concatenate([y, u, lam])
    return np.linalg.norm(r) / np.linalg.norm(kkt_rhs(b))


def objective(M, b, c, beta, y, u):
    return 0.5 * y @ (M @ y) - b @ y + 0.5 * c + 0.5 * beta * u @ (M @ u)


def state_solve(M, K, u):
    return spla.spsolve(sp.csc_matrix(K), M @ u)


def adjoint_solve(M, K, b, y):
    return spla.spsolve(sp.csc_matrix(K.T), b - M @ y)


def reduced_objective(M, K, b, c, beta, u):
    y = state_solve(M, K, u)
    return objective(M, b, c, beta, y, u)


def reduced_gradient(M, K, b, beta, u):
    """dJ/du of u -> J(y(u), u) with K y = M u: beta M u - M lam."""
    y = state_solve(M, K, u)
    lam = adjoint_solve(M, K, b, y)
    return beta * (M @ u) - M @ lam, y, lam


def fast_diag_solve(M1s, K1s, beta, b):
    """KKT solve when M = M1 (x) M2 (x) M3 and K = K1(x)M2(x)M3 + M1(x)K2(x)M3 + M1(x)M2(x)K3.

    Generalised eigenvectors V_d (K_d V_d = M_d V_d Lambda_d, V_d^T M_d V_d = I)
    turn M into the identity and K into the diagonal Lambda_1 (+) Lambda_2 (+)
    Lambda_3; per eigenmode the KKT system is the 3 x 3 system
    [[1,0,k],[0,beta,-1],[k,-1,0]] with solution y = bt / (1 + beta k^2),
    lam = beta k y, u = lam / beta.
    """
    Vs, lams = [], []
    for M1, K1 in zip(M1s, K1s):
        lam, V = sla.eigh(K1, M1)
        Vs.append(V)
        lams.append(lam)
    n = [V.shape[0] for V in Vs]
    B = b.reshape(n)
    bt = np.einsum("ia,jb,kc,ijk->abc", Vs[0], Vs[1], Vs[2], B)
    kap = lams[0][:, None, None] + lams[1][None, :, None] + lams[2][None, None, :]
    yt = bt / (1.0 + beta * kap ** 2)
    lt = beta * kap * yt
    ut = lt / beta
    back = lambda T: np.einsum("ia,jb,kc,abc->ijk", Vs[0], Vs[1], Vs[2], T).ravel()
    return back(yt), back(ut), back(lt)


def reduced_solve(M_apply, K_apply, Minv_apply, beta, b, tol=1e-12, precond=None, maxit=10000):
    """Stationary KKT solve through the reduced (Schur) system, by conjugate gradients.

    Rows 2 and 3 of eq. KKTSystem (one time step) give lam = beta u and
    M u = K y, so u = M^{-1} K y; row 1, M y + K^T lam = b with K = K^T, then
    reads

        S y = (M + beta K M^{-1} K) y = b,

    with S symmetric positive definite.  CG on S (preconditioned by `precond`,
    a callable approximating S^{-1}; None for plain CG) until
    ||b - S y|| <= tol ||b||, then u = M^{-1} K y and lam = beta u.  The
    operators are callables on flat vectors.  Returns (y, u, lam, iterations).
    """
    b = np.asarray(b, dtype=np.float64)
    S = lambda v: M_apply(v) + beta * K_apply(Minv_apply(K_apply(v)))
    P = precond if precond is not None else (lambda v: v)
    y = np.zeros_like(b)
    r = b.copy()
    z = P(r)
    d = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    it = 0
    while np.linalg.norm(r) > tol * nb and it < maxit:
        Sd = S(d)
        alpha = rz / (d @ Sd)
        y += alpha * d
        r -= alpha * Sd
        z = P(r)
        rz_new = r @ z
        d = z + (rz_new / rz) * d
        rz = rz_new
        it += 1
    u = Minv_apply(K_apply(y))
    return y, u, beta * u, it


def kron_schur_preconditioner(M1s, G1s, beta):
    """Approximate inverse of S = M + beta K M^{-1} K for CG (changes the
    iteration count, not the solution of `reduced_solve`).

    With M ~ M_1 (x) M_2 (x) M_3 and K ~ sum_d G_d (x) M_e (x) M_f the
    generalised eigenvectors V_d of (G_d, M_d) diagonalise both, and
    S ~ V (I + beta Kappa^2) V^T with Kappa = Lambda_1 (+) Lambda_2 (+)
    Lambda_3 (the same algebra as `fast_diag_solve`; exact on the unit cube).
    """
    Vs, lams = [], []
    for M1, G1 in zip(M1s, G1s):
        lam, V = sla.eigh(G1, M1)
        Vs.append(V)
        lams.append(lam)
    n = [V.shape[0] for V in Vs]
    kap = lams[0][:, None, None] + lams[1][None, :, None] + lams[2][None, None, :]
    dinv = 1.0 / (1.0 + beta * kap ** 2)

    def apply(r):
        R = r.reshape(n)
        T = np.einsum("ia,jb,kc,ijk->abc", Vs[0], Vs[1], Vs[2], R, optimize=True) * dinv
        return np.einsum("ia,jb,kc,abc->ijk", Vs[0], Vs[1], Vs[2], T, optimize=True).ravel()
    return apply
