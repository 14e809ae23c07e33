"""Pins of the oracle's geometry map, Jacobian and weights."""
import math

import numpy as np
import pytest

from oracle.geometry import map_and_jacobian, weights_from_jacobian
from paper_1811_06797_gb300 import workloads as wl


def _eval(geo, pts):
    return map_and_jacobian(geo.kind, geo.degree, geo.knots, geo.homogeneous(), geo.twist, pts)


def _pts(m=200, seed=0):
    return np.random.default_rng(seed).uniform(0.0, 1.0, size=(m, 3))


def test_unit_cube_identity():
    x = _pts()
    G, J = _eval(wl.unit_cube(), x)
    assert np.allclose(G, x, atol=1e-15)
    om, Q, det = weights_from_jacobian(J)
    assert np.allclose(om, 1.0) and np.allclose(Q, np.eye(3))


def test_affine_box_closed_form():
    A = np.array([[2.0, 0.3, 0.1], [0.0, 1.5, -0.2], [0.1, 0.0, 0.7]])
    geo = wl.affine_box(A, shift=(1.0, -2.0, 0.5))
    x = _pts()
    G, J = _eval(geo, x)
    assert np.allclose(G, x @ A.T + np.array([1.0, -2.0, 0.5]))
    om, Q, _ = weights_from_jacobian(J)
    assert np.allclose(om, abs(np.linalg.det(A)))
    assert np.allclose(Q, np.linalg.inv(A.T @ A) * abs(np.linalg.det(A)))


def test_annulus_image_and_weights():
    geo = wl.quarter_annulus()
    x = _pts()
    G, J = _eval(geo, x)
    r = np.hypot(G[:, 0], G[:, 1])
    # direction 2 is radial and linear: r = 1 + xhat_2 exactly for the NURBS circle
    assert np.allclose(r, 1.0 + x[:, 1], atol=1e-14)
    assert np.all(G[:, 0] >= -1e-15) and np.all(G[:, 1] >= -1e-15)
    assert np.allclose(G[:, 2], x[:, 2])
    om, Q, det = weights_from_jacobian(J)
    # metric is diagonal: off-diagonal Q vanish, omega = r |c'(s)|
    assert np.allclose(Q[:, 0, 1], 0, atol=1e-13) and np.allclose(Q[:, 0, 2], 0, atol=1e-13)
    assert np.allclose(Q[:, 1, 2], 0, atol=1e-13)
    speed = np.linalg.norm(J[:, :2, 0], axis=1) / r
    assert np.allclose(om, r * speed)


@pytest.mark.parametrize("geo", [wl.quarter_annulus(), wl.quarter_annulus(twist=math.pi / 4),
                                 wl.random_volume()])
def test_jacobian_matches_finite_differences(geo):
    x = np.random.default_rng(3).uniform(0.05, 0.95, size=(60, 3))
    _, J = _eval(geo, x)
    h = 1e-6
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        Gp, _ = _eval(geo, x + e)
        Gm, _ = _eval(geo, x - e)
        assert np.allclose((Gp - Gm) / (2 * h), J[:, :, b], atol=1e-7)


def test_twist_preserves_determinant():
    x = _pts(seed=5)
    _, J0 = _eval(wl.quarter_annulus(), x)
    _, J1 = _eval(wl.quarter_annulus(twist=math.pi / 4), x)
    assert np.allclose(np.linalg.det(J0), np.linalg.det(J1), rtol=1e-13)
    # but the metric, hence Q, changes
    _, Q0, _ = weights_from_jacobian(J0)
    _, Q1, _ = weights_from_jacobian(J1)
    assert np.max(np.abs(Q0 - Q1)) > 1e-2


def test_random_volume_is_valid():
    geo = wl.random_volume()
    x = _pts(2000, seed=9)
    _, J = _eval(geo, x)
    assert np.all(np.linalg.det(J) > 0.5)
