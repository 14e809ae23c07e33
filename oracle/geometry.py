"""Oracle: NURBS volume map, its Jacobian and the geometry weights.

Test infrastructure only (see the package header).

G(xhat) = C : B(xhat) (Sec. 2, eq. geometryMapping) with the NURBS
quotient of Sec. 2 (rational map with weights w_i).  The twisted geometry is
R(twist * z) G(xhat), a rotation about e_z by an angle proportional to the
physical z coordinate (analytic composition, not a NURBS).

Weights (Sec. 2 after eq. stiffness, and Sec. 3):
  omega = |det J|,  Q = (J^T J)^{-1} omega,  J_ab = d G_a / d xhat_b.
The reading J^T J (metric tensor in parametric coordinates) is the one for
which  int_Omega grad u . grad v dx = int (Q grad^ u) . grad^ v dxhat.

Pins: volume of the unit cube, parallelepipeds and the (twisted) quarter
annulus; omega and Q of an affine map in closed form; the annulus Jacobian
against finite differences of G; manufactured Poisson solutions converge
at the optimal rate (tests/test_oracle_assembly.py).
"""
from __future__ import annotations

import numpy as np

from .bspline import basis_all

GEO_NURBS_TWIST = 1


def _rot(theta):
    c, s = np.cos(theta), np.sin(theta)
    return c, s


def map_and_jacobian(kind, degree, knots, hw, twist, xh):
    """G and J at parametric points xh of shape (P, 3).

    hw: homogeneous control net (n1, n2, n3, 4) = (w x, w y, w z, w).
    Returns G (P, 3) and J (P, 3, 3) with J[:, a, b] = dG_a / dxhat_b.
    """
    xh = np.asarray(xh, dtype=np.float64)
    B, dB = [], []
    for d in range(3):
        v, dv = basis_all(knots[d], degree[d], xh[:, d])
        B.append(v)
        dB.append(dv)
    # homogeneous point A(xhat) and its parametric derivatives
    A = np.einsum("pi,pj,pk,ijkm->pm", B[0], B[1], B[2], hw)
    dA = np.stack([
        np.einsum("pi,pj,pk,ijkm->pm", dB[0], B[1], B[2], hw),
        np.einsum("pi,pj,pk,ijkm->pm", B[0], dB[1], B[2], hw),
        np.einsum("pi,pj,pk,ijkm->pm", B[0], B[1], dB[2], hw),
    ], axis=-1)                                   # (P, 4, 3)
    w = A[:, 3]
    G = A[:, :3] / w[:, None]
    # quotient rule: dG/dxhat_b = (dA_{0:3}/dxhat_b - G dw/dxhat_b) / w
    J = (dA[:, :3, :] - G[:, :, None] * dA[:, 3:4, :]) / w[:, None, None]
    if kind == GEO_NURBS_TWIST:
        theta = twist * G[:, 2]
        c, s = _rot(theta)
        x, y = G[:, 0], G[:, 1]
        Gt = np.stack([c * x - s * y, s * x + c * y, G[:, 2]], axis=1)
        # d/dxhat_b [R(theta) G] = R dG/dxhat_b + R'(theta) G * twist * dz/dxhat_b
        Jt = np.empty_like(J)
        dz = J[:, 2, :]
        Jt[:, 0, :] = c[:, None] * J[:, 0, :] - s[:, None] * J[:, 1, :] \
            + twist * (-s * x - c * y)[:, None] * dz
        Jt[:, 1, :] = s[:, None] * J[:, 0, :] + c[:, None] * J[:, 1, :] \
            + twist * (c * x - s * y)[:, None] * dz
        Jt[:, 2, :] = J[:, 2, :]
        return Gt, Jt
    return G, J


def weights_from_jacobian(J):
    """omega = |det J| and Q = (J^T J)^{-1} |det J| at each point."""
    det = np.linalg.det(J)
    omega = np.abs(det)
    JtJ = np.einsum("pab,pac->pbc", J, J)
    Q = np.linalg.inv(JtJ) * omega[:, None, None]
    return omega, Q, det


def grid_points(xs):
    """Tensor grid of the three 1-D point sets, flattened in C order."""
    g = np.meshgrid(xs[0], xs[1], xs[2], indexing="ij")
    return np.stack([a.ravel() for a in g], axis=1)
