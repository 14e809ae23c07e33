"""Pins of the oracle's 3-D assembly (mass, stiffness, load)."""
import math
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest
import scipy.sparse.linalg as spla
from scipy.interpolate import BSpline

from oracle.assemble import (Discretisation, assemble_band, band_to_csr, dense_bruteforce,
                             sampled_rows, sample_weights)
from oracle.bspline import basis_all
from paper_1811_06797_gb300 import workloads as wl


def disc_of(space):
    return Discretisation(space.degree, space.knots, space.nquad)


def cardinal(m, x, deriv=0):
    """Cardinal B-spline of order m (degree m-1) at x, or its deriv-th derivative, exactly."""
    x = Fraction(x)
    s = Fraction(0)
    e = m - 1 - deriv
    for k in range(m + 1):
        t = x - k
        if t > 0:
            s += (-1) ** k * comb(m, k) * t ** e
    return s / factorial(e)


def exact_1d(knots, p):
    """1-D mass and stiffness via scipy B-splines and a 20-point numpy Gauss rule per span."""
    n = len(knots) - p - 1
    spl = BSpline(knots, np.eye(n), p)
    dspl = spl.derivative()
    t, w = np.polynomial.legendre.leggauss(20)
    M = np.zeros((n, n))
    K = np.zeros((n, n))
    u = np.unique(knots)
    for a, b in zip(u[:-1], u[1:]):
        x = 0.5 * (a + b) + 0.5 * (b - a) * t
        g = 0.5 * (b - a) * w
        V = spl(x)
        D = dspl(x)
        M += V.T @ (g[:, None] * V)
        K += D.T @ (g[:, None] * D)
    return M, K


@pytest.mark.parametrize("p,E", [(2, 5), (3, 4)])
def test_unit_cube_kronecker_structure(p, E):
    sp_ = wl.uniform_space(p, E)
    disc = disc_of(sp_)
    Mb, Kb, _ = assemble_band(wl.unit_cube(), disc)
    M = band_to_csr(Mb).toarray()
    K = band_to_csr(Kb).toarray()
    M1, K1 = exact_1d(sp_.knots[0], p)
    Mk = np.kron(M1, np.kron(M1, M1))
    Kk = np.kron(K1, np.kron(M1, M1)) + np.kron(M1, np.kron(K1, M1)) + np.kron(M1, np.kron(M1, K1))
    assert np.abs(M - Mk).max() < 1e-15 * 10
    assert np.abs(K - Kk).max() < 1e-12 * np.abs(Kk).max()


@pytest.mark.parametrize("p", [2, 3])
def test_1d_interior_entries_are_cardinal_autocorrelations(p):
    E = 12
    k = wl.open_uniform_knots(p, E)
    M1, K1 = exact_1d(k, p)
    h = 1.0 / E
    n = M1.shape[0]
    m = 2 * p + 2
    for i in range(p, n - p - 1 - p):
        for o in range(0, p + 1):
            mref = h * float(cardinal(m, p + 1 + o))
            kref = -float(cardinal(m, p + 1 + o, deriv=2)) / h
            assert abs(M1[i, i + o] - mref) < 1e-15
            assert abs(K1[i, i + o] - kref) < 1e-12 * abs(K1[i, i])
    # the textbook values for p = 2: 66/120, 26/120, 1/120
    if p == 2:
        assert [cardinal(6, 3 + o) for o in range(3)] == [Fraction(66, 120), Fraction(26, 120),
                                                           Fraction(1, 120)]


GEOS = {
    "cube": wl.unit_cube(),
    "box": wl.affine_box(np.array([[1.5, 0.2, 0.0], [0.1, 0.8, 0.3], [0.0, -0.2, 1.1]])),
    "annulus": wl.quarter_annulus(),
    "twisted": wl.quarter_annulus(twist=math.pi / 4),
    "random": wl.random_volume(),
}


@pytest.mark.parametrize("name", ["cube", "box", "annulus", "twisted"])
def test_volume_and_neumann_kernel(name):
    geo = GEOS[name]
    # a rational omega is not integrated exactly: many points per element for the annulus
    nq = 3 if name in ("cube", "box") else 9
    disc = disc_of(wl.uniform_space(2, 3, nq))
    Mb, Kb, _ = assemble_band(geo, disc)
    M = band_to_csr(Mb)
    K = band_to_csr(Kb)
    one = np.ones(M.shape[0])
    assert abs(one @ (M @ one) - geo.volume) < 1e-11 * geo.volume
    assert np.abs(K @ one).max() < 1e-12 * abs(K).max()


@pytest.mark.parametrize("name", ["annulus", "twisted", "random"])
def test_symmetry_and_definiteness(name):
    disc = disc_of(wl.uniform_space(2, 4))
    Mb, Kb, _ = assemble_band(GEOS[name], disc)
    M = band_to_csr(Mb).toarray()
    K = band_to_csr(Kb).toarray()
    assert np.abs(M - M.T).max() < 1e-14 * np.abs(M).max()
    assert np.abs(K - K.T).max() < 1e-12 * np.abs(K).max()
    np.linalg.cholesky(M)                                  # SPD
    ev = np.linalg.eigvalsh(K)
    assert ev[0] > -1e-12 * ev[-1] and ev[1] > 1e-8 * ev[-1]   # PSD, one-dimensional kernel
    Mi = band_to_csr(Mb, interior=True).toarray()
    Ki = band_to_csr(Kb, interior=True).toarray()
    np.linalg.cholesky(Mi)
    np.linalg.cholesky(Ki)                                 # Dirichlet: SPD


@pytest.mark.parametrize("name", ["twisted", "random"])
def test_band_assembly_equals_bruteforce(name):
    geo = GEOS[name]
    disc = disc_of(wl.uniform_space(2, 4))
    tgt = wl.Target(wl.TARGET_GAUSS, (0.9, 0.9, 0.5), 0.1)
    Mb, Kb, b = assemble_band(geo, disc, tgt)
    Md, Kd, bd = dense_bruteforce(geo, disc, tgt)
    assert np.abs(band_to_csr(Mb).toarray() - Md).max() < 1e-14 * np.abs(Md).max() * 10
    assert np.abs(band_to_csr(Kb).toarray() - Kd).max() < 1e-13 * np.abs(Kd).max()
    assert np.abs(b.ravel() - bd).max() < 1e-14 * np.abs(bd).max() * 10


def test_sampled_load_equals_band():
    from oracle.assemble import sampled_load
    geo = GEOS["twisted"]
    disc = disc_of(wl.uniform_space(3, 4))
    tgt = wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1)
    _, _, b = assemble_band(geo, disc, tgt)
    rows = np.array([(0, 0, 0), (1, 2, 3), (6, 6, 6), (3, 0, 5)])
    got = sampled_load(geo, disc, tgt, rows)
    assert np.allclose(got, [b[tuple(r)] for r in rows], rtol=1e-13, atol=1e-17)


def test_sampled_rows_equal_band():
    geo = GEOS["twisted"]
    disc = disc_of(wl.uniform_space(3, 5))
    Mb, Kb, _ = assemble_band(geo, disc)
    rng = np.random.default_rng(1)
    rows = np.stack([rng.integers(0, n, 12) for n in disc.n], axis=1)
    rows[0] = (0, 0, 0)
    rows[1] = tuple(n - 1 for n in disc.n)
    Mr, Kr = sampled_rows(geo, disc, rows)
    for s, r in enumerate(rows):
        assert np.allclose(Mr[s], Mb[tuple(r)], atol=1e-17, rtol=1e-12)
        assert np.allclose(Kr[s], Kb[tuple(r)], atol=1e-14, rtol=1e-12)


# --- manufactured Poisson solutions: -Lap u = f, u = 0 on the boundary -------------------

def _manufactured(name):
    import sympy as sy
    x, y, z = sy.symbols("x y z", real=True)
    if name == "cube":
        u = sy.sin(sy.pi * x) * sy.sin(sy.pi * y) * sy.sin(sy.pi * z)
    else:
        r = sy.sqrt(x ** 2 + y ** 2)
        th = sy.atan2(y, x)
        tw = sy.pi / 4 if name == "twisted" else 0
        u = (r - 1) * (2 - r) * sy.sin(2 * (th - tw * z)) * sy.sin(sy.pi * z)
    f = -(sy.diff(u, x, 2) + sy.diff(u, y, 2) + sy.diff(u, z, 2))
    U = sy.lambdify((x, y, z), u, "numpy")
    F = sy.lambdify((x, y, z), f, "numpy")
    return (lambda P: U(P[:, 0], P[:, 1], P[:, 2])), (lambda P: F(P[:, 0], P[:, 1], P[:, 2]))


def _l2_error(geo, disc, coef, ufun):
    xs, gs = disc.gauss_grid()
    V = [basis_all(disc.knots[d], disc.degree[d], xs[d], nderiv=0)[0] for d in range(3)]
    uh = np.einsum("ai,bj,ck,ijk->abc", V[0], V[1], V[2], coef)
    G, om, _, _ = sample_weights(geo, disc)
    ue = ufun(G.reshape(-1, 3)).reshape(uh.shape)
    W = om * np.einsum("a,b,c->abc", *gs)
    return math.sqrt(np.sum(W * (uh - ue) ** 2))


@pytest.mark.parametrize("name", ["cube", "annulus", "twisted"])
def test_manufactured_poisson_converges(name):
    pytest.importorskip("sympy")
    geo = GEOS[name]
    ufun, ffun = _manufactured(name)
    errs = []
    for E in (3, 6):
        disc = disc_of(wl.uniform_space(2, E))
        _, Kb, b = assemble_band(geo, disc, ffun)
        K = band_to_csr(Kb, interior=True)
        y = spla.spsolve(K.tocsc(), b[1:-1, 1:-1, 1:-1].ravel())
        coef = np.zeros(disc.n)
        coef[1:-1, 1:-1, 1:-1] = y.reshape(tuple(n - 2 for n in disc.n))
        errs.append(_l2_error(geo, disc, coef, ufun))
    rate = math.log2(errs[0] / errs[1])
    assert rate > 2.4, (errs, rate)       # optimal L2 rate p + 1 = 3
