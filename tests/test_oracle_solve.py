"""Pins of the oracle's large-grid KKT route (oracle/solve.py): low-rank
operators, reduced-system CG, exact or iterative M^{-1}, against the sparse
direct solve of the 3-D assembled system."""
import math

import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.kkt import kkt_solve
from oracle.solve import interior_operators, solve_kkt
from paper_1811_06797_gb300 import workloads as wl


@pytest.mark.parametrize("geo,p,E,beta", [(wl.quarter_annulus(), 3, 4, 1e-4),
                                          (wl.quarter_annulus(twist=math.pi / 4), 2, 5, 1e-6),
                                          (wl.random_volume(), 2, 4, 1e-4)])
def test_low_rank_reduced_route_equals_direct_solve(geo, p, E, beta):
    work = wl.small(geo, p, E, wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=beta,
                    tol=1e-13)
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, b = assemble_band(work.geometry, disc, work.target)
    M, K = band_to_csr(Mb, True), band_to_csr(Kb, True)
    yd, ud, ld = kkt_solve(M, K, beta, b[1:-1, 1:-1, 1:-1].ravel())
    Mt, Kt, diag, bl = interior_operators(work.space, work.geometry, work.target, work.tol)
    assert np.linalg.norm(bl - b[1:-1, 1:-1, 1:-1].ravel()) < 1e-11 * np.linalg.norm(bl)
    y, u, lam, it = solve_kkt(Mt, Kt, diag, bl, beta, tol=1e-13)
    for a, c in ((y, yd), (u, ud), (lam, ld)):
        assert np.linalg.norm(a - c) < 1e-8 * np.linalg.norm(c)


def test_interpolated_route_operators_equal_sampled_route_on_an_affine_box():
    """With a constant Jacobian every weight is a constant, which the spline
    interpolation reproduces exactly: the interpolated route's interior
    operators and load must equal the sampled route's (the Kronecker matrices
    compared densely on a 3-element grid)."""
    from oracle.lowrank import kron_matrix
    from oracle.solve import interior_operators_interp
    geo = wl.affine_box(np.array([[1.0, 0.2, 0.0], [0.1, 0.9, 0.3], [0.0, 0.2, 1.3]]))
    space = wl.uniform_space(2, 3)
    target = wl.Target(wl.TARGET_SINPROD)
    Ms, Ks, _, bs = interior_operators(space, geo, target, 1e-14)
    Mi, Ki, _, bi = interior_operators_interp(space, geo, target, 1e-14)
    for A, B in ((Ms, Mi), (Ks, Ki)):
        As, Ai = kron_matrix(A).toarray(), kron_matrix(B).toarray()
        assert np.linalg.norm(As - Ai) < 1e-12 * np.linalg.norm(As)
    # the load density sin(pi x) sin(pi y) sin(pi z) o G is not polynomial:
    # only the interpolation error of degree 5 on 3 elements separates the loads
    assert np.linalg.norm(bs - bi) < 1e-3 * np.linalg.norm(bs)
    assert np.linalg.norm(bs - bi) > 0.0
