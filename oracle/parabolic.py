"""Oracle: the parabolic (time-dependent) KKT system.

Test infrastructure only (see the package header).

Sec. 4, eq. timeDiscrete: implicit Euler in time with N_t steps of size tau
and the rectangle rule in the objective give the discrete problem

    min  sum_k tau/2 [ (y_k - yhat_k)^T M (y_k - yhat_k) + beta u_k^T M u_k ]
    s.t. (M y_k - M y_{k-1}) / tau + K y_k = M u_k,   k = 1..N_t,  y_0 = 0,

and its optimality conditions form eq. KKTSystem,

    [ tau MM      0          KK^T   ] [y  ]   [b]
    [ 0        tau beta MM  -tau MM ] [u  ] = [0]
    [ KK      -tau MM        0      ] [lam]   [0]

with MM = I_{N_t} (x) M, KK = I_{N_t} (x) tau K + C (x) M, C the lower
bidiagonal time difference (1 on the diagonal, -1 below) and
b = tau MM yhat.  Vectors are stacked in time, y = [y_1; ...; y_{N_t}]
(time the slow index).  As in the stationary oracle the right-hand side
block b is an input: b_k = tau M yhat_k for a desired state yhat.

`state_stepping` and `adjoint_stepping` are the forward and backward
implicit Euler sweeps written from the discrete problem itself (not from the
Kronecker form): they pin the assembled system, together with the reduced
gradient (central differences of the objective along the state equation)
and the one-step case, which is the stationary system with K + M / tau
(tests/test_oracle_parabolic.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def time_difference(nt):
    """C of eq. KKTSystem: ones on the diagonal, minus ones below it."""
    return sp.diags([np.ones(nt), -np.ones(nt - 1)], [0, -1], shape=(nt, nt), format="csr")


def space_time_operators(M, K, tau, nt):
    """MM = I (x) M and KK = I (x) tau K + C (x) M (Sec. 4, eqs. M_kron / K_kron)."""
    I = sp.identity(nt, format="csr")
    MM = sp.kron(I, M, format="csr")
    KK = sp.kron(I, tau * K, format="csr") + sp.kron(time_difference(nt), M, format="csr")
    return MM, KK


def kkt_matrix_parabolic(M, K, tau, beta, nt):
    MM, KK = space_time_operators(M, K, tau, nt)
    Z = None
    return sp.bmat([[tau * MM, Z, KK.T], [Z, tau * beta * MM, -tau * MM], [KK, -tau * MM, Z]],
                   format="csc")


def kkt_rhs_parabolic(b):
    """[b; 0; 0] for b of shape (N_t, N)."""
    b = np.asarray(b, dtype=np.float64).ravel()
    return np.concatenate([b, np.zeros_like(b), np.zeros_like(b)])


def kkt_solve_parabolic(M, K, tau, beta, b):
    """Sparse direct solve (SuperLU); b, y, u, lam of shape (N_t, N)."""
    b = np.asarray(b, dtype=np.float64)
    nt, N = b.shape
    z = spla.spsolve(kkt_matrix_parabolic(M, K, tau, beta, nt), kkt_rhs_parabolic(b))
    n = nt * N
    return z[:n].reshape(nt, N), z[n:2 * n].reshape(nt, N), z[2 * n:].reshape(nt, N)


def kkt_apply_parabolic(M, K, tau, beta, y, u, lam):
    """The KKT operator on (y, u, lam), each (N_t, N); returns the three rows."""
    nt, N = y.shape
    A = kkt_matrix_parabolic(M, K, tau, beta, nt)
    r = A @ np.concatenate([y.ravel(), u.ravel(), lam.ravel()])
    n = nt * N
    return r[:n].reshape(nt, N), r[n:2 * n].reshape(nt, N), r[2 * n:].reshape(nt, N)


def kkt_residual_parabolic(M, K, tau, beta, b, y, u, lam):
    """||rhs - A z||_2 / ||rhs||_2."""
    ry, ru, rl = kkt_apply_parabolic(M, K, tau, beta, y, u, lam)
    rhs = kkt_rhs_parabolic(b)
    r = rhs - np.concatenate([ry.ravel(), ru.ravel(), rl.ravel()])
    return np.linalg.norm(r) / np.linalg.norm(rhs)


def state_stepping(M, K, tau, u):
    """Implicit Euler for the state: (M + tau K) y_k = M y_{k-1} + tau M u_k, y_0 = 0."""
    A = sp.csc_matrix(M + tau * K)
    lu = spla.splu(A)
    y = np.zeros_like(u)
    prev = np.zeros(u.shape[1])
    for k in range(u.shape[0]):
        y[k] = lu.solve(M @ prev + tau * (M @ u[k]))
        prev = y[k]
    return y


def adjoint_stepping(M, K, tau, b, y):
    """The adjoint backwards in time, from the y-rows of the optimality conditions:
    (M + tau K^T) lam_k = M lam_{k+1} + b_k - tau M y_k, lam_{N_t + 1} = 0."""
    lu = spla.splu(sp.csc_matrix(M + tau * K.T))
    lam = np.zeros_like(y)
    nxt = np.zeros(y.shape[1])
    for k in range(y.shape[0] - 1, -1, -1):
        lam[k] = lu.solve(M @ nxt + b[k] - tau * (M @ y[k]))
        nxt = lam[k]
    return lam


def objective_parabolic(M, tau, beta, yhat, y, u):
    """The rectangle-rule objective of eq. timeDiscrete in coefficients."""
    J = 0.0
    for k in range(y.shape[0]):
        e = y[k] - yhat[k]
        J += 0.5 * tau * (e @ (M @ e) + beta * u[k] @ (M @ u[k]))
    return J


def reduced_objective_parabolic(M, K, tau, beta, yhat, u):
    return objective_parabolic(M, tau, beta, yhat, state_stepping(M, K, tau, u), u)


def reduced_gradient_parabolic(M, K, tau, beta, yhat, u):
    """dJ/du_k along the state equation: tau beta M u_k - tau M lam_k, with lam from
    the adjoint sweep for b = tau M yhat."""
    y = state_stepping(M, K, tau, u)
    b = np.stack([tau * (M @ yh) for yh in yhat])
    lam = adjoint_stepping(M, K, tau, b, y)
    g = np.stack([tau * beta * (M @ u[k]) - tau * (M @ lam[k]) for k in range(u.shape[0])])
    return g, y, lam
