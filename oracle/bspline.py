"""Oracle: knot vectors, Gauss-Legendre quadrature, Cox-de Boor recursion.

Test infrastructure only (see the package header).

Pins (tests/test_oracle_bspline.py): Gauss rule integrates monomials up to
degree 2q-1 exactly and matches numpy's leggauss; basis values match
scipy.interpolate.BSpline and form a partition of unity; derivatives match
central finite differences; Greville abscissae reproduce the identity.
"""
from __future__ import annotations

import numpy as np


def check_open_knots(knots: np.ndarray, degree: int) -> int:
    """Validate an open knot vector (Sec. 2, eq. knotVector); return n = #basis.

    End knots 0 and 1 repeated degree+1 times, nondecreasing, interior
    multiplicity at most degree.
    """
    k = np.asarray(knots, dtype=np.float64)
    p = degree
    n = len(k) - p - 1
    if n < p + 1:
        raise ValueError("too few knots")
    if np.any(np.diff(k) < 0):
        raise ValueError("knots must be nondecreasing")
    if not (np.all(k[:p + 1] == 0.0) and np.all(k[n:] == 1.0)):
        raise ValueError("end knots must be 0 and 1 with multiplicity degree+1")
    inner = k[p + 1:n]
    if len(inner):
        vals, counts = np.unique(inner, return_counts=True)
        if np.any(counts > p):
            raise ValueError("interior knot multiplicity exceeds degree")
        if np.any((vals <= 0.0) | (vals >= 1.0)):
            raise ValueError("interior knots must lie in (0, 1)")
    return n


def legendre_and_derivative(q: int, t: np.ndarray):
    """P_q(t) and P_q'(t) by the three-term recurrence."""
    p0 = np.ones_like(t)
    p1 = t.copy()
    if q == 0:
        return p0, np.zeros_like(t)
    for k in range(2, q + 1):
        p0, p1 = p1, ((2 * k - 1) * t * p1 - (k - 1) * p0) / k
    dp = q * (t * p1 - p0) / (t * t - 1.0)
    return p1, dp


def gauss_legendre(q: int):
    """Nodes and weights of the q-point Gauss-Legendre rule on [-1, 1].

    Newton iteration on P_q from the Chebyshev-like initial guess
    cos(pi (k - 1/4) / (q + 1/2)); weights 2 / ((1 - t^2) P_q'(t)^2).
    """
    k = np.arange(1, q + 1)
    t = np.cos(np.pi * (k - 0.25) / (q + 0.5))
    for _ in range(100):
        p, dp = legendre_and_derivative(q, t)
        dt = p / dp
        t = t - dt
        if np.max(np.abs(dt)) < 1e-16:
            break
    p, dp = legendre_and_derivative(q, t)
    w = 2.0 / ((1.0 - t * t) * dp * dp)
    order = np.argsort(t)
    return t[order], w[order]


def elements(knots: np.ndarray) -> np.ndarray:
    """Nonempty knot spans [a, b] as an (E, 2) array (the elements)."""
    u = np.unique(np.asarray(knots, dtype=np.float64))
    return np.stack([u[:-1], u[1:]], axis=1)


def element_quadrature(knots: np.ndarray, q: int):
    """Gauss points and weights on every element: arrays of shape (E, q)."""
    t, w = gauss_legendre(q)
    el = elements(knots)
    a, b = el[:, :1], el[:, 1:]
    x = 0.5 * (a + b) + 0.5 * (b - a) * t[None, :]
    g = 0.5 * (b - a) * w[None, :]
    return x, g


def basis_all(knots: np.ndarray, degree: int, x: np.ndarray, nderiv: int = 1):
    """All n B-splines of the given degree (and first derivatives) at points x.

    Cox-de Boor recursion of Sec. 2:
      beta_{i,0}(x) = 1 if xhat_i <= x < xhat_{i+1} else 0,
      beta_{i,j}(x) = (x - xhat_i) / (xhat_{i+j} - xhat_i) beta_{i,j-1}(x)
                    + (xhat_{i+j+1} - x) / (xhat_{i+j+1} - xhat_{i+1}) beta_{i+1,j-1}(x),
    with 0/0 := 0.  At x = 1 the last nonempty span is taken as closed.
    Derivative: beta'_{i,p} = p [beta_{i,p-1} / (xhat_{i+p} - xhat_i)
                                  - beta_{i+1,p-1} / (xhat_{i+p+1} - xhat_{i+1})].
    Returns (values, derivatives), each of shape (len(x), n).
    """
    k = np.asarray(knots, dtype=np.float64)
    p = degree
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    m = len(k) - 1                      # number of zero-degree functions
    n = len(k) - p - 1
    last = np.max(np.nonzero(k[:-1] < k[1:])[0])   # last nonempty span
    b = np.zeros((len(x), m))
    for i in range(m):
        if k[i] < k[i + 1]:
            inside = (k[i] <= x) & (x < k[i + 1])
            if i == last:
                inside |= (x == k[i + 1])
            b[:, i] = inside
    lower = None
    for j in range(1, p + 1):
        if j == p:
            lower = b.copy()
        nb = np.zeros((len(x), m - j))
        for i in range(m - j):
            d1 = k[i + j] - k[i]
            d2 = k[i + j + 1] - k[i + 1]
            t1 = (x - k[i]) / d1 * b[:, i] if d1 > 0 else 0.0
            t2 = (k[i + j + 1] - x) / d2 * b[:, i + 1] if d2 > 0 else 0.0
            nb[:, i] = t1 + t2
        b = nb
    values = b[:, :n]
    if nderiv == 0:
        return values, None
    if p == 0:
        return values, np.zeros_like(values)
    der = np.zeros((len(x), n))
    for i in range(n):
        d1 = k[i + p] - k[i]
        d2 = k[i + p + 1] - k[i + 1]
        t1 = lower[:, i] / d1 if d1 > 0 else 0.0
        t2 = lower[:, i + 1] / d2 if d2 > 0 else 0.0
        der[:, i] = p * (t1 - t2)
    return values, der
