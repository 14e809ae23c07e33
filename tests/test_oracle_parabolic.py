"""Pins of the parabolic oracle (Sec. 4, eqs. timeDiscrete and KKTSystem).

The assembled space-time KKT system is checked against what the discrete
problem itself fixes, written without the Kronecker form: the forward
implicit Euler sweep of the state equation, the backward sweep of the
adjoint, u = lam / beta, a zero reduced gradient of the rectangle-rule
objective at the solution (central differences), the gradient formula at
any control, and the single-step case, which is the stationary system with
stiffness K + M / tau."""
import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.kkt import kkt_solve
from oracle.parabolic import (adjoint_stepping, kkt_residual_parabolic, kkt_solve_parabolic,
                              reduced_gradient_parabolic, reduced_objective_parabolic,
                              state_stepping, time_difference)
from paper_1811_06797_gb300 import workloads as wl


def _mk(E=3, p=2):
    work = wl.small(wl.quarter_annulus(), p, E, beta=1e-3)
    s = work.space
    disc = Discretisation(s.degree, s.knots, s.nquad)
    Mb, Kb, _ = assemble_band(work.geometry, disc, work.target)
    return band_to_csr(Mb, interior=True), band_to_csr(Kb, interior=True)


def _yhat(nt, N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((nt, N))


def test_time_difference_is_the_implicit_euler_stencil():
    C = time_difference(4).toarray()
    # (C (x) I) y at step k is y_k - y_{k-1}, with y_0 = 0
    y = np.array([1.0, 3.0, 6.0, 10.0])
    assert np.array_equal(C @ y, np.array([1.0, 2.0, 3.0, 4.0]))


@pytest.mark.parametrize("nt,tau,beta", [(4, 0.25, 1e-2), (6, 0.1, 1e-4)])
def test_time_stepping_reproduces_the_kkt_solution(nt, tau, beta):
    M, K = _mk()
    N = M.shape[0]
    yhat = _yhat(nt, N, nt)
    b = np.stack([tau * (M @ yh) for yh in yhat])
    y, u, lam = kkt_solve_parabolic(M, K, tau, beta, b)
    assert kkt_residual_parabolic(M, K, tau, beta, b, y, u, lam) < 1e-12
    # the state equation swept forward from the control
    ys = state_stepping(M, K, tau, u)
    assert np.linalg.norm(ys - y) <= 1e-10 * np.linalg.norm(y)
    # the adjoint swept backward from the state
    ls = adjoint_stepping(M, K, tau, b, y)
    assert np.linalg.norm(ls - lam) <= 1e-10 * np.linalg.norm(lam)
    # the control rows: beta u = lam
    assert np.linalg.norm(beta * u - lam) <= 1e-10 * np.linalg.norm(lam)


def test_kkt_solution_has_zero_reduced_gradient():
    M, K = _mk()
    nt, tau, beta = 5, 0.2, 1e-2
    N = M.shape[0]
    yhat = _yhat(nt, N, 11)
    b = np.stack([tau * (M @ yh) for yh in yhat])
    _, u, _ = kkt_solve_parabolic(M, K, tau, beta, b)
    rng = np.random.default_rng(3)
    J0 = reduced_objective_parabolic(M, K, tau, beta, yhat, u)
    for _ in range(3):
        v = rng.standard_normal(u.shape)
        v /= np.linalg.norm(v)
        eps = 1e-3
        Jp = reduced_objective_parabolic(M, K, tau, beta, yhat, u + eps * v)
        Jm = reduced_objective_parabolic(M, K, tau, beta, yhat, u - eps * v)
        # a quadratic: the central difference is the exact directional derivative
        slope = (Jp - Jm) / (2 * eps)
        curv = (Jp + Jm - 2 * J0) / eps ** 2
        assert curv > 0.0
        assert abs(slope) <= 1e-8 * (abs(J0) / np.linalg.norm(u) + curv)


def test_reduced_gradient_matches_finite_differences():
    M, K = _mk()
    nt, tau, beta = 4, 0.25, 1e-2
    N = M.shape[0]
    yhat = _yhat(nt, N, 5)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((nt, N))
    g, _, _ = reduced_gradient_parabolic(M, K, tau, beta, yhat, u)
    for _ in range(3):
        v = rng.standard_normal(u.shape)
        eps = 1e-3
        fd = (reduced_objective_parabolic(M, K, tau, beta, yhat, u + eps * v)
              - reduced_objective_parabolic(M, K, tau, beta, yhat, u - eps * v)) / (2 * eps)
        assert abs(fd - np.sum(g * v)) <= 1e-7 * (abs(fd) + 1e-12)


def test_one_step_is_the_stationary_system_with_shifted_stiffness():
    # N_t = 1: tau [[M, 0, K + M/tau], [0, beta M, -M], [K + M/tau, -M, 0]]
    M, K = _mk()
    tau, beta = 0.3, 1e-3
    N = M.shape[0]
    b = _yhat(1, N, 2)
    y, u, lam = kkt_solve_parabolic(M, K, tau, beta, b)
    ys, us, ls = kkt_solve(M, K + M / tau, beta, b[0] / tau)
    for a, c in ((y[0], ys), (u[0], us), (lam[0], ls)):
        assert np.linalg.norm(a - c) <= 1e-10 * np.linalg.norm(c)
