"""Pins of the oracle's weight-interpolation route (oracle/interp.py, Sec. 3
eqs. weightEquationSystem / weightEquationSolve)."""
import numpy as np
import pytest

from oracle.assemble import Discretisation
from oracle.bspline import basis_all
from oracle.interp import greville, interp_knots, node_to_gauss, weight_tts_interp
from oracle.lowrank import tt_full, weight_tts
from paper_1811_06797_gb300 import workloads as wl


def disc_of(p, E):
    s = wl.uniform_space(p, E)
    return Discretisation(s.degree, s.knots, s.nquad)


def full(cores):
    return None if cores is None else tt_full(cores)


def cubic_stretch():
    """x = xhat + 0.3 xhat^2 + 0.2 xhat^3 (a cubic Bezier in direction 1), y = yhat,
    z = zhat: |det J| = 1 + 0.6 xhat + 0.6 xhat^2, a quadratic."""
    k3 = np.array([0, 0, 0, 0, 1, 1, 1, 1], float)
    k1 = np.array([0, 0, 1, 1], float)
    bx = [0.0, 1.0 / 3.0, 1.0 / 3.0 * 2 + 0.1, 1.5]      # power-to-Bernstein coefficients
    c = np.zeros((4, 2, 2, 3))
    for i in range(4):
        for j in range(2):
            for m in range(2):
                c[i, j, m] = (bx[i], j, m)
    return wl.Geometry(wl.GEO_NURBS, (3, 1, 1), (k3, k1, k1.copy()), c, np.ones((4, 2, 2)))


def test_collocation_rows_and_node_map_reproduce_constants():
    for p, E in ((1, 3), (2, 5), (3, 4)):
        d = disc_of(p, E)
        pt = 2 * p + 1
        kt = interp_knots(d.knots[0], pt)
        Bt, _ = basis_all(kt, pt, greville(kt, pt), nderiv=0)
        assert np.allclose(Bt.sum(axis=1), 1.0, atol=1e-14)
        L = node_to_gauss(d.knots[0], pt, d.gauss_grid()[0][0])
        assert np.allclose(L @ np.ones(L.shape[1]), 1.0, atol=1e-12)


@pytest.mark.parametrize("name", ["cube", "box", "cubic"])
def test_polynomial_weights_are_reproduced_exactly(name):
    geo = {"cube": wl.unit_cube(), "box": wl.affine_box(np.array([[1.0, 0.2, 0.0],
                                                                   [0.1, 0.9, 0.3],
                                                                   [0.0, 0.2, 1.3]])),
           "cubic": cubic_stretch()}[name]
    d = disc_of(2, 4)
    a = weight_tts_interp(geo, d, 1e-14)
    b = weight_tts(geo, d, 1e-14)
    wa, wb = full(a["omega"]), full(b["omega"])
    assert np.linalg.norm(wa - wb) < 1e-12 * np.linalg.norm(wb)
    if name != "cubic":          # constant Jacobian: Q constant too
        for k in range(3):
            for l in range(k, 3):
                qa, qb = full(a[(k, l)]), full(b[(k, l)])
                if qb is None:
                    assert qa is None or np.abs(qa).max() < 1e-13
                else:
                    assert np.linalg.norm(qa - qb) < 1e-12 * np.linalg.norm(qb)


def test_interpolation_error_falls_at_rate_h_to_pt_plus_one():
    # the annulus weight is rational: the interpolant at the Gauss points
    # converges to the sampled weight at the spline rate h^(pt+1)
    geo = wl.quarter_annulus()
    errs = []
    for E in (3, 6):
        d = disc_of(1, E)
        wa = full(weight_tts_interp(geo, d, 1e-14, pt=3)["omega"])
        wb = full(weight_tts(geo, d, 1e-14)["omega"])
        errs.append(np.linalg.norm(wa - wb) / np.linalg.norm(wb))
    assert errs[1] < errs[0] / 8, errs          # rate 2^4 = 16 with some slack
    assert errs[0] > 1e-12                      # not exact: the rate is measurable
