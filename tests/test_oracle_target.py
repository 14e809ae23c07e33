"""Pins of the desired state yhat and of the load vector built from it.

The objective of Sec. 1 / Sec. 4 measures the distance to a desired state
yhat; the stationary reading of eq. KKTSystem feeds it in through the load
vector b_i = int yhat(G(xhat)) beta_i omega dxhat.  These pins fix
`target_values` / `evaluate_target` at points where the definition gives the
value outright, and the assembled load vector through integrals with a
closed form or a library quadrature: by the partition of unity the entries of
b over the full (not Dirichlet-reduced) space add up to int_Omega yhat dx.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.special import erf

from oracle.assemble import Discretisation, assemble_band, evaluate_target, target_values
from paper_1811_06797_gb300 import workloads as wl


def disc_of(space):
    return Discretisation(space.degree, space.knots, space.nquad)


def test_gaussian_target_at_its_centre_and_one_width_away():
    c = np.array([0.3, -0.2, 0.7])
    w = 0.1
    rng = np.random.default_rng(5)
    d = rng.standard_normal((6, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    pts = np.concatenate([c[None], c + math.sqrt(w) * d, c + 2 * math.sqrt(w) * d])
    v = target_values(wl.TARGET_GAUSS, [*c, w], pts)
    assert v[0] == 1.0
    assert np.allclose(v[1:7], math.exp(-1.0), rtol=1e-15, atol=0)
    assert np.allclose(v[7:], math.exp(-4.0), rtol=1e-14, atol=0)


def test_sine_product_target_vanishes_on_the_faces_and_peaks_in_the_middle():
    rng = np.random.default_rng(6)
    faces = rng.random((12, 3))
    for k in range(3):
        faces[4 * k:4 * k + 2, k] = 0.0
        faces[4 * k + 2:4 * k + 4, k] = 1.0
    v = target_values(wl.TARGET_SINPROD, [0, 0, 0, 1], faces)
    assert np.abs(v).max() < 1e-15
    mid = target_values(wl.TARGET_SINPROD, [0, 0, 0, 1], np.array([[0.5, 0.5, 0.5],
                                                                     [0.25, 0.5, 0.5]]))
    assert mid[0] == 1.0
    assert abs(mid[1] - math.sqrt(0.5)) < 1e-15


def test_evaluate_target_uses_the_workload_description():
    tgt = wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1)
    x = np.array([wl.ANNULUS_CENTROID, (1.0, 1.0, 0.0)])
    v = evaluate_target(tgt, x)
    c = np.array(wl.ANNULUS_CENTROID)
    assert v[0] == 1.0
    assert abs(v[1] - math.exp(-np.sum((x[1] - c) ** 2) / 0.1)) < 1e-16
    assert np.allclose(evaluate_target(lambda p: p[:, 0] * 2.0, x), 2.0 * x[:, 0])


def _load_sum(geo, target, p=1, nelem=8, nquad=8):
    _, _, b = assemble_band(geo, disc_of(wl.uniform_space(p, nelem, nquad)), target)
    return float(b.sum())


def test_load_of_the_sine_product_on_the_unit_cube():
    # int_[0,1]^3 prod sin(pi x_k) dx = (2/pi)^3
    got = _load_sum(wl.unit_cube(), wl.Target(wl.TARGET_SINPROD))
    assert abs(got - (2.0 / math.pi) ** 3) < 1e-12


def test_load_of_the_gaussian_on_the_unit_cube():
    # int_0^1 exp(-(x - c)^2 / w) dx = sqrt(pi w)/2 (erf((1 - c)/sqrt w) + erf(c/sqrt w))
    c, w = (0.3, 0.6, 0.45), 0.1
    exact = 1.0
    for ck in c:
        exact *= 0.5 * math.sqrt(math.pi * w) * (erf((1 - ck) / math.sqrt(w)) + erf(ck / math.sqrt(w)))
    got = _load_sum(wl.unit_cube(), wl.Target(wl.TARGET_GAUSS, c, w))
    assert abs(got - exact) < 1e-11 * exact


def test_annulus_centroid_is_the_first_moment_over_the_volume():
    # int x over the quarter annulus r in [1, 2], z in [0, 1] is 7/3 (and so is
    # int y); with the volume 3 pi / 4 the centroid is 28 / (9 pi)
    geo = wl.quarter_annulus()
    mx = _load_sum(geo, lambda p: p[:, 0], p=2, nelem=4, nquad=9)
    my = _load_sum(geo, lambda p: p[:, 1], p=2, nelem=4, nquad=9)
    mz = _load_sum(geo, lambda p: p[:, 2], p=2, nelem=4, nquad=9)
    assert abs(mx - 7.0 / 3.0) < 1e-11 and abs(my - 7.0 / 3.0) < 1e-11
    assert abs(mx / geo.volume - wl.ANNULUS_CENTROID[0]) < 1e-11
    assert abs(mz / geo.volume - 0.5) < 1e-11


@pytest.mark.parametrize("twist", [0.0, math.pi / 4])
def test_load_of_the_gaussian_on_the_annulus_matches_library_quadrature(twist):
    # the physical integral in cylindrical coordinates, z-part in closed form
    # (the twist rotates each z-slice about e_z, which maps the annulus onto
    # itself only as a set of slices: the integrand is evaluated at the rotated
    # points, and the volume element r dr dtheta dz is unchanged)
    c = np.array(wl.ANNULUS_CENTROID)
    w = 0.1

    def slice_integral(z):
        th0 = twist * z

        def f(theta, r):
            x = r * math.cos(theta + th0) - c[0]
            y = r * math.sin(theta + th0) - c[1]
            return math.exp(-(x * x + y * y) / w) * r
        val, _ = integrate.dblquad(f, 1.0, 2.0, 0.0, math.pi / 2, epsabs=1e-14, epsrel=1e-13)
        return val * math.exp(-(z - c[2]) ** 2 / w)

    if twist == 0.0:
        zpart = 0.5 * math.sqrt(math.pi * w) * (erf((1 - c[2]) / math.sqrt(w)) + erf(c[2] / math.sqrt(w)))
        exact = slice_integral(c[2]) * zpart
    else:
        exact, _ = integrate.quad(slice_integral, 0.0, 1.0, epsabs=1e-14, epsrel=1e-12, limit=200)
    geo = wl.quarter_annulus(twist=twist)
    got = _load_sum(geo, wl.Target(wl.TARGET_GAUSS, tuple(c), w), p=1, nelem=8, nquad=8)
    assert abs(got - exact) < 1e-10 * exact
