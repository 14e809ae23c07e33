"""GPU parity of the block-AMEn KKT solve (a6-a8) against the oracle's direct solves."""
import math

import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.kkt import fast_diag_solve, kkt_residual, kkt_solve
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch
from test_oracle_kkt import _exact_1d_interior

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _oracle_system(work):
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, b = assemble_band(work.geometry, disc, work.target)
    return band_to_csr(Mb, True), band_to_csr(Kb, True), b[1:-1, 1:-1, 1:-1].ravel()


def _solve(env, work, **opts):
    ctx, torch, iga = env
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    info = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, y, u, lam, **opts)
    return info, y.cpu().numpy(), u.cpu().numpy(), lam.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    ("cube", wl.small(wl.unit_cube(), 2, 6, beta=1e-2, tol=1e-12)),
    ("cube_b6", wl.small(wl.unit_cube(), 2, 8, beta=1e-6, tol=1e-12)),
    ("annulus", wl.small(wl.quarter_annulus(), 3, 7,
                         wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-4, tol=1e-12)),
    ("twisted", wl.small(wl.quarter_annulus(twist=math.pi / 4), 2, 9,
                         wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-3, tol=1e-12)),
    # TT-matrix operators with weight ranks > 1 (random cubic volume)
    ("random", wl.small(wl.random_volume(), 2, 6, wl.Target(wl.TARGET_SINPROD), beta=1e-4,
                        tol=1e-12)),
]


@pytest.mark.parametrize("name,work", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("trunc", [0, 1], ids=["pivoted", "svd"])
def test_solve_matches_direct(env, name, work, prec, trunc):
    info, y, u, lam = _solve(env, work, tol=1e-10, precision=prec, truncation=trunc)
    assert info["converged"], info
    M, K, b = _oracle_system(work)
    # residual of the GPU solution measured with the oracle's 3-D assembled matrices
    assert kkt_residual(M, K, work.beta, b, y, u, lam) < 1e-9
    yo, uo, lo = kkt_solve(M, K, work.beta, b)
    for got, ref in ((y, yo), (u, uo), (lam, lo)):
        assert _rel(got, ref) < 1e-6, (name, _rel(got, ref))


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_config1_against_fast_diagonalisation(env, prec):
    work = wl.config(1)
    info, y, u, lam = _solve(env, work, tol=1e-10, precision=prec)
    assert info["converged"], info
    _, _, b = _oracle_system(work)
    M1, K1 = _exact_1d_interior(work.space.knots[0], 2)
    yf, uf, lf = fast_diag_solve([M1] * 3, [K1] * 3, work.beta, b)
    for got, ref in ((y, yf), (u, uf), (lam, lf)):
        assert _rel(got, ref) < 1e-6


def test_solve_reports_no_convergence(env):
    work = CASES[2][1]
    info, *_ = _solve(env, work, tol=1e-12, refine_max=0, max_sweeps=1)
    assert not info["converged"] and info["residual"] > 1e-12


def test_random_volume_truncated_operator(env):
    """Weights truncated at 1e-6: the solve matches the direct solve of the
    oracle's exact matrices up to the truncation error of the operator."""
    ctx, torch, iga = env
    work = wl.small(wl.random_volume(), 2, 6, wl.Target(wl.TARGET_SINPROD), beta=1e-3, tol=1e-6)
    info, y, u, lam = _solve(env, work, tol=1e-9, precision=0)
    assert info["converged"], info
    M, K, b = _oracle_system(work)
    yo, uo, lo = kkt_solve(M, K, work.beta, b)
    assert _rel(y, yo) < 1e-4 and _rel(lam, lo) < 1e-4
    # and the operator really has TT ranks above one
    Mop, Kop, _ = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    assert max(Mop.info()["R"]) > 1
