"""Pins of the oracle's KKT solve, objective and reduced gradient."""
import math

import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.kkt import (fast_diag_solve, kkt_residual, kkt_solve, objective, reduced_gradient,
                        reduced_objective)
from paper_1811_06797_gb300 import workloads as wl


def _exact_1d_interior(knots, p):
    n = len(knots) - p - 1
    spl = BSpline(knots, np.eye(n), p)
    dspl = spl.derivative()
    t, w = np.polynomial.legendre.leggauss(12)
    M = np.zeros((n, n))
    K = np.zeros((n, n))
    u = np.unique(knots)
    for a, b in zip(u[:-1], u[1:]):
        x = 0.5 * (a + b) + 0.5 * (b - a) * t
        g = 0.5 * (b - a) * w
        V, D = spl(x), dspl(x)
        M += V.T @ (g[:, None] * V)
        K += D.T @ (g[:, None] * D)
    return M[1:-1, 1:-1], K[1:-1, 1:-1]


def _system(work):
    s = work.space
    disc = Discretisation(s.degree, s.knots, s.nquad)
    Mb, Kb, b = assemble_band(work.geometry, disc, work.target)
    M = band_to_csr(Mb, interior=True)
    K = band_to_csr(Kb, interior=True)
    return M, K, b[1:-1, 1:-1, 1:-1].ravel()


@pytest.mark.parametrize("E,beta", [(6, 1e-2), (6, 1e-6), (10, 1e-6)])
def test_unit_cube_direct_equals_fast_diagonalisation(E, beta):
    # the fast-diagonalisation solve is the unit-cube KKT reference at the full
    # 16-element size; here it is pinned to SuperLU where that finishes quickly
    work = wl.small(wl.unit_cube(), 2, E, beta=beta)
    M, K, b = _system(work)
    y, u, lam = kkt_solve(M, K, beta, b)
    M1, K1 = _exact_1d_interior(work.space.knots[0], 2)
    yf, uf, lf = fast_diag_solve([M1] * 3, [K1] * 3, beta, b)
    # both solves leave residuals at rounding level; the solutions then agree up to
    # the conditioning of the KKT matrix (u = lam / beta amplifies at small beta)
    assert kkt_residual(M, K, beta, b, y, u, lam) < 1e-12
    assert kkt_residual(M, K, beta, b, yf, uf, lf) < 1e-11
    for a, c in ((y, yf), (u, uf), (lam, lf)):
        assert np.linalg.norm(a - c) < 1e-6 * np.linalg.norm(c)


def test_kkt_solution_is_optimal():
    work = wl.small(wl.quarter_annulus(), 2, 4,
                    wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-3)
    M, K, b = _system(work)
    y, u, lam = kkt_solve(M, K, work.beta, b)
    assert np.linalg.norm(work.beta * u - lam) < 1e-10 * np.linalg.norm(lam)
    assert np.linalg.norm(K @ y - M @ u) < 1e-10 * np.linalg.norm(M @ u)
    g, _, _ = reduced_gradient(M, K, b, work.beta, u)
    assert np.linalg.norm(g) < 1e-9 * np.linalg.norm(work.beta * (M @ u))


def test_reduced_gradient_matches_finite_differences():
    work = wl.small(wl.quarter_annulus(twist=math.pi / 4), 2, 3,
                    wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-2)
    M, K, b = _system(work)
    rng = np.random.default_rng(4)
    u = rng.standard_normal(len(b))
    v = rng.standard_normal(len(b))
    g, _, _ = reduced_gradient(M, K, b, work.beta, u)
    h = 1e-6
    fd = (reduced_objective(M, K, b, 1.0, work.beta, u + h * v)
          - reduced_objective(M, K, b, 1.0, work.beta, u - h * v)) / (2 * h)
    assert abs(fd - g @ v) < 1e-7 * max(1.0, abs(fd))


def test_objective_definition():
    # J(y,u) = 1/2 ||y - yhat||_M^2 + beta/2 ||u||_M^2 with yhat itself in the space:
    # then b = M yhat, c = yhat^T M yhat and J(yhat, 0) = 0
    work = wl.small(wl.unit_cube(), 2, 3)
    M, K, _ = _system(work)
    yh = np.random.default_rng(0).standard_normal(M.shape[0])
    b = M @ yh
    c = yh @ b
    assert abs(objective(M, b, c, 0.3, yh, np.zeros_like(yh))) < 1e-14


@pytest.mark.parametrize("geo,beta", [(wl.quarter_annulus(), 1e-3),
                                      (wl.quarter_annulus(twist=math.pi / 4), 1e-5),
                                      (wl.random_volume(), 1e-4)])
def test_reduced_cg_equals_direct_solve(geo, beta):
    # eliminating u and lam (rows 2 and 3 of eq. KKTSystem) and solving the
    # Schur system by CG must reproduce SuperLU on the full KKT matrix
    import scipy.sparse.linalg as spla
    from oracle.kkt import reduced_solve
    work = wl.small(geo, 2, 4, wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=beta)
    M, K, b = _system(work)
    y, u, lam = kkt_solve(M, K, beta, b)
    lu = spla.splu(M.tocsc())
    yr, ur, lr, it = reduced_solve(lambda v: M @ v, lambda v: K @ v, lu.solve, beta, b, tol=1e-13)
    assert it > 3
    for a, c in ((yr, y), (ur, u), (lr, lam)):
        assert np.linalg.norm(a - c) < 1e-9 * np.linalg.norm(c)


def test_reduced_cg_with_kronecker_preconditioner_on_the_unit_cube():
    # on the unit cube the Kronecker preconditioner is the exact inverse of S,
    # so preconditioned CG stops after one step at the fast-diagonalisation
    # solution
    from oracle.kkt import kron_schur_preconditioner, reduced_solve
    E, beta = 6, 1e-6
    work = wl.small(wl.unit_cube(), 2, E, beta=beta)
    M, K, b = _system(work)
    M1, K1 = _exact_1d_interior(work.space.knots[0], 2)
    P = kron_schur_preconditioner([M1] * 3, [K1] * 3, beta)
    n1 = M1.shape[0]
    M1i = np.linalg.inv(M1)
    Mi = lambda v: np.einsum("ia,jb,kc,abc->ijk", M1i, M1i, M1i, v.reshape((n1,) * 3)).ravel()
    y, u, lam, it = reduced_solve(lambda v: M @ v, lambda v: K @ v, Mi, beta, b, tol=1e-12,
                                  precond=P)
    yf, uf, lf = fast_diag_solve([M1] * 3, [K1] * 3, beta, b)
    assert it <= 2
    for a, c in ((y, yf), (u, uf), (lam, lf)):
        assert np.linalg.norm(a - c) < 1e-8 * np.linalg.norm(c)
