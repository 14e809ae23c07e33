"""Oracle: the weights interpolated in a spline space S~ (Sec. 3, eqs.
weightEquationSystem and weightEquationSolve).

Test infrastructure only (see the package header).

Each weight (omega and the entries of Q, and the load density yhat(G) omega)
is represented as a tensor-product spline of degree pt on the break points of
the discretisation, w(xhat) = sum_j W_j Bt_j(xhat).  Its coefficients solve
the collocation system at the Greville abscissae xi of S~,

    (Bt_1 (x) Bt_2 (x) Bt_3) vec(W) = vec(w(xi)),   Bt_d[i, j] = Bt_j(xi_i),

which on a TT of the node values w(xi) is one solve per direction and core
(eq. weightEquationSolve).  The univariate integrals then use the
interpolant at the Gauss points of the discretisation: every core is mapped
by E_d Bt_d^{-1}, E_d[g, j] = Bt_j(x_g), and multiplied by the Gauss
weights g_d, which gives a TT of the same kind as lowrank.weight_tts (the
sampled weights times the Gauss weights) and feeds the same univariate
assembly.

The degree: the paper states Dp+1 (Sec. 3) and 2p+1 (Sec. 6); the default
here is 2p+1.

Pins (tests/test_oracle_interp.py): the node values of a weight that is a
polynomial of degree <= pt in each direction are reproduced exactly at the
Gauss points (unit cube, affine box, a trilinear map's |det J|); the
interpolation error of the curved geometries falls at rate h^(pt+1) under
refinement; the collocation matrix has the partition-of-unity row sums.
"""
from __future__ import annotations

import numpy as np

from .assemble import evaluate_target
from .bspline import basis_all
from .geometry import grid_points, map_and_jacobian, weights_from_jacobian
from .lowrank import tt_svd


def interp_knots(knots, pt):
    """Open knot vector of degree pt on the break points of `knots`."""
    br = np.unique(np.asarray(knots, dtype=np.float64))
    return np.concatenate([np.zeros(pt), br, np.ones(pt)])


def greville(knots, pt):
    n = len(knots) - pt - 1
    return np.array([knots[i + 1:i + pt + 1].mean() for i in range(n)])


def node_to_gauss(knots, pt, xg):
    """E Bt^{-1}: the interpolant's values at the points xg from its node values."""
    kt = interp_knots(knots, pt)
    xi = greville(kt, pt)
    Bt, _ = basis_all(kt, pt, xi, nderiv=0)
    E, _ = basis_all(kt, pt, xg, nderiv=0)
    return E @ np.linalg.inv(Bt)


def weight_tts_interp(geo, disc, tol, target=None, pt=None):
    """TT cores of the interpolated omega g, q_kl g (k <= l) and the load
    density at the Gauss points, in the layout of lowrank.weight_tts."""
    pt = 2 * max(disc.degree) + 1 if pt is None else pt
    xs = [greville(interp_knots(k, pt), pt) for k in disc.knots]
    pts = grid_points(xs)
    G, J = map_and_jacobian(geo.kind, geo.degree, geo.knots, geo.homogeneous(), geo.twist, pts)
    omega, Q, _ = weights_from_jacobian(J)
    shp = tuple(len(x) for x in xs)
    omega = omega.reshape(shp)
    Q = Q.reshape(shp + (3, 3))
    xg, gs = disc.gauss_grid()
    maps = [node_to_gauss(k, pt, x) * g[:, None] for k, x, g in zip(disc.knots, xg, gs)]

    def to_gauss(cores):
        if cores is None:
            return None
        return [np.einsum("gi,aib->agb", L, c) for L, c in zip(maps, cores)]

    out = {"omega": to_gauss(tt_svd(omega, tol))}
    qn = np.linalg.norm(Q)
    for k in range(3):
        for l in range(k, 3):
            out[(k, l)] = to_gauss(tt_svd(Q[..., k, l], tol, norm=qn))
    if target is not None:
        f = evaluate_target(target, G).reshape(shp) * omega
        out["load"] = to_gauss(tt_svd(f, tol))
    return out
