"""Pins of the oracle's knot, quadrature and Cox-de Boor routines."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle.bspline import basis_all, check_open_knots, gauss_legendre, element_quadrature


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 8])
def test_gauss_exact_monomials(q):
    t, w = gauss_legendre(q)
    for k in range(2 * q):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.sum(w * t ** k) - exact) < 1e-14
    # first non-exact degree really is inexact (a wrong rule with extra exactness would be odd)
    k = 2 * q
    assert abs(np.sum(w * t ** k) - 2.0 / (k + 1)) > 1e-8


@pytest.mark.parametrize("q", [2, 3, 4, 7])
def test_gauss_matches_library(q):
    t, w = gauss_legendre(q)
    tl, wl = np.polynomial.legendre.leggauss(q)
    assert np.allclose(t, tl, atol=1e-15, rtol=0) and np.allclose(w, wl, atol=1e-15, rtol=0)


def test_element_quadrature_integrates_on_spans():
    knots = np.array([0, 0, 0, 0.25, 0.5, 0.5, 1, 1, 1.0])
    x, g = element_quadrature(knots, 3)
    assert x.shape == (3, 3)
    assert abs(g.sum() - 1.0) < 1e-15
    assert abs(np.sum(g * x ** 5) - 1.0 / 6.0) < 1e-15


KNOTS = [
    (1, np.array([0, 0, 0.5, 1, 1.0])),
    (2, np.array([0, 0, 0, 0.2, 0.5, 0.5, 0.7, 1, 1, 1.0])),
    (3, np.array([0, 0, 0, 0, 0.1, 0.4, 0.4, 0.4, 0.8, 1, 1, 1, 1.0])),
    (3, np.concatenate([np.zeros(3), np.linspace(0, 1, 9), np.ones(3)])),
]


@pytest.mark.parametrize("p,knots", KNOTS)
def test_basis_matches_scipy(p, knots):
    n = check_open_knots(knots, p)
    x = np.concatenate([np.linspace(0, 1, 57), [0.2, 0.5, 0.4, 1.0]])
    v, dv = basis_all(knots, p, x)
    ref = BSpline(knots, np.eye(n), p, extrapolate=False)
    rv = ref(x)
    rd = ref.derivative()(x)
    # scipy leaves x == 1 undefined (nan) on the half-open convention: use the left limit
    at_end = x == 1.0
    rv[at_end] = BSpline(knots, np.eye(n), p)(1.0 - 1e-15)
    rd[at_end] = BSpline(knots, np.eye(n), p).derivative()(1.0 - 1e-15)
    assert np.allclose(v, rv, atol=1e-13)
    assert np.allclose(dv, rd, atol=1e-9 * max(1.0, np.abs(rd).max()))


@pytest.mark.parametrize("p,knots", KNOTS)
def test_partition_of_unity_and_fd(p, knots):
    x = np.linspace(0.013, 0.987, 41)
    v, dv = basis_all(knots, p, x)
    assert np.allclose(v.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(dv.sum(axis=1), 0.0, atol=1e-11)
    assert np.all(v >= -1e-15)
    # derivative by central differences away from knots
    h = 1e-6
    interior = [xx for xx in x if np.min(np.abs(knots - xx)) > 1e-3]
    interior = np.array(interior)
    vp, _ = basis_all(knots, p, interior + h, nderiv=0)
    vm, _ = basis_all(knots, p, interior - h, nderiv=0)
    _, d0 = basis_all(knots, p, interior)
    assert np.allclose((vp - vm) / (2 * h), d0, atol=1e-6 * max(1.0, np.abs(d0).max()))


def test_support_and_count():
    p, knots = KNOTS[1]
    n = check_open_knots(knots, p)
    x = np.linspace(0, 1, 201)
    v, _ = basis_all(knots, p, x)
    assert v.shape[1] == n
    for i in range(n):
        outside = (x < knots[i]) | (x > knots[i + p + 1])
        assert np.all(v[outside, i] == 0.0)


@pytest.mark.parametrize("bad", [
    (2, np.array([0, 0, 0.5, 1, 1, 1.0])),               # start multiplicity 2 < p+1
    (2, np.array([0, 0, 0, 0.6, 0.4, 1, 1, 1.0])),        # decreasing
    (1, np.array([0, 0, 0.5, 0.5, 1, 1.0])),              # interior multiplicity > p
])
def test_bad_knots_rejected(bad):
    p, k = bad
    with pytest.raises(ValueError):
        check_open_knots(k, p)
