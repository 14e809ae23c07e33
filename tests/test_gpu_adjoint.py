"""GPU parity of the adjoint / gradient path (a9) against the oracle and finite differences."""
import math

import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.kkt import reduced_gradient, reduced_objective
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch

pytestmark = pytest.mark.gpu

TGT = wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1)


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _oracle(work):
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, b = assemble_band(work.geometry, disc, work.target)
    return band_to_csr(Mb, True), band_to_csr(Kb, True), b[1:-1, 1:-1, 1:-1].ravel()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("which", ["M", "K"])
def test_spd_solve_matches_direct(env, which):
    ctx, torch, iga = env
    import scipy.sparse.linalg as spla
    work = wl.small(wl.quarter_annulus(twist=math.pi / 4), 3, 6, TGT, beta=1e-3, tol=1e-12)
    M, K, _ = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    Mo, Ko, _ = _oracle(work)
    N = Mo.shape[0]
    b = np.random.default_rng(0).standard_normal(N)
    x = torch.zeros(N, dtype=torch.float64, device="cuda")
    A = M if which == "M" else K
    info = iga.iga_spd_solve(ctx, A, M, K, torch.tensor(b, device="cuda"), x, tol=1e-12)
    ref = spla.spsolve((Mo if which == "M" else Ko).tocsc(), b)
    assert _rel(x.cpu().numpy(), ref) < 1e-9
    if which == "M":
        assert info["iters"] <= 2          # the preconditioner is M^-1 itself


@pytest.mark.parametrize("name,geo", [("annulus", wl.quarter_annulus()),
                                      ("twisted", wl.quarter_annulus(twist=math.pi / 4))])
def test_reduced_gradient_matches_oracle(env, name, geo):
    ctx, torch, iga = env
    work = wl.small(geo, 2, 5, TGT, beta=1e-3, tol=1e-12)
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    Mo, Ko, bo = _oracle(work)
    N = Mo.shape[0]
    u = np.random.default_rng(1).standard_normal(N)
    ut = torch.tensor(u, device="cuda")
    g, y, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    J = iga.iga_reduced_gradient(ctx, M, K, load, work.beta, ut, g, y, lam, tol=1e-13)
    go, yo, lo = reduced_gradient(Mo, Ko, bo, work.beta, u)
    assert _rel(g.cpu().numpy(), go) < 1e-8
    assert _rel(y.cpu().numpy(), yo) < 1e-9 and _rel(lam.cpu().numpy(), lo) < 1e-9
    Jo = reduced_objective(Mo, Ko, bo, 0.0, work.beta, u)
    assert abs(J[0] - Jo) < 1e-9 * abs(Jo)


def test_reduced_gradient_finite_differences(env):
    ctx, torch, iga = env
    work = wl.small(wl.quarter_annulus(twist=math.pi / 4), 3, 6, TGT, beta=1e-2, tol=1e-12)
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    rng = np.random.default_rng(2)
    u = torch.tensor(rng.standard_normal(N), device="cuda")
    v = torch.tensor(rng.standard_normal(N), device="cuda")
    g, y, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    iga.iga_reduced_gradient(ctx, M, K, load, work.beta, u, g, y, lam, tol=1e-13)
    h = 1e-6
    Jp = iga.iga_reduced_gradient(ctx, M, K, load, work.beta, u + h * v, y.clone(), y, lam, 1e-13)[0]
    Jm = iga.iga_reduced_gradient(ctx, M, K, load, work.beta, u - h * v, y.clone(), y, lam, 1e-13)[0]
    fd = (Jp - Jm) / (2 * h)
    an = float(torch.dot(g, v))
    assert abs(fd - an) < 1e-6 * max(1.0, abs(an))


def test_weight_gradient_finite_differences(env):
    ctx, torch, iga = env
    from paper_1811_06797_gb300.autograd import geometry_factors, operators_from_factors
    work = wl.small(wl.quarter_annulus(twist=math.pi / 4), 2, 5, TGT, beta=1e-2, tol=1e-12)
    w, load = geometry_factors(ctx, work.geometry, work.space, work.target, work.tol)
    M, K = operators_from_factors(ctx, work.space, w)
    N = int(np.prod(M.info()["n"]))
    rng = np.random.default_rng(3)
    u = torch.tensor(rng.standard_normal(N), device="cuda")
    g, y, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    iga.iga_reduced_gradient(ctx, M, K, load, work.beta, u, g, y, lam, tol=1e-13)
    gw = torch.empty_like(w)
    iga.iga_weight_gradient(ctx, work.space, M, K, work.beta, y, u, lam, gw)

    def J_of(wp):
        Mp, Kp = operators_from_factors(ctx, work.space, wp)
        gg, yy, ll = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
        return iga.iga_reduced_gradient(ctx, Mp, Kp, load, work.beta, u, gg, yy, ll, 1e-13)[0]

    active = [c for c in range(7) if bool(torch.any(w[c] != 0))]
    assert 0 in active and 3 in active                    # omega and q13 (twist coupling)
    for c in active:
        v = torch.zeros_like(w)
        v[c] = torch.tensor(rng.standard_normal(w.shape[1]), device="cuda") * w[c].abs().max()
        h = 1e-6
        fd = (J_of(w + h * v) - J_of(w - h * v)) / (2 * h)
        an = float((gw * v).sum())
        assert abs(fd - an) < 1e-5 * max(1e-8, abs(an)), (c, fd, an)


def test_autograd_function(env):
    ctx, torch, iga = env
    from paper_1811_06797_gb300.autograd import geometry_factors, objective
    work = wl.small(wl.quarter_annulus(), 2, 4, TGT, beta=1e-2, tol=1e-12)
    w, load = geometry_factors(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod([len(k) - 3 - 2 for k in work.space.knots]))
    u = torch.tensor(np.random.default_rng(4).standard_normal(N), device="cuda", requires_grad=True)
    wr = w.clone().requires_grad_(True)
    J = objective(ctx, work.space, load, work.beta, u, wr)
    J.backward()
    assert u.grad is not None and wr.grad is not None
    # against the oracle's reduced gradient with the same control
    Mo, Ko, bo = _oracle(work)
    go, _, _ = reduced_gradient(Mo, Ko, bo, work.beta, u.detach().cpu().numpy())
    assert _rel(u.grad.cpu().numpy(), go) < 1e-8
    # directional derivative in w by central differences through the Function
    v = torch.randn_like(w) * (w != 0)
    h = 1e-6
    with torch.no_grad():
        fd = (objective(ctx, work.space, load, work.beta, u, w + h * v)
              - objective(ctx, work.space, load, work.beta, u, w - h * v)) / (2 * h)
    an = float((wr.grad * v).sum())
    assert abs(float(fd) - an) < 1e-5 * max(1e-8, abs(an))


def test_config4_batch_gradients(env):
    """Twisted annulus, degree 3, 128 elements: 8 seeded controls smoothed by 3 mass solves."""
    ctx, torch, iga = env
    work = wl.config(4)
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    n = M.info()["n"]
    N = int(np.prod(n))
    U = wl.random_controls(n, work.extra["seeds"]).reshape(8, N)
    u = torch.tensor(U, device="cuda")
    for _ in range(3):                      # smoothing: u <- M^-1 u, rescaled to unit RMS
        for s in range(8):
            x = torch.zeros(N, dtype=torch.float64, device="cuda")
            iga.iga_spd_solve(ctx, M, M, K, u[s].contiguous(), x, tol=1e-12)
            u[s] = x / torch.sqrt(torch.mean(x * x))
    g, y, lam = (torch.empty((8, N), dtype=torch.float64, device="cuda") for _ in range(3))
    J = iga.iga_reduced_gradient(ctx, M, K, load, work.beta, u, g, y, lam, tol=1e-12)
    assert np.all(np.isfinite(J))
    # central differences (h = 1e-6) along a random direction for two of the controls
    rng = np.random.default_rng(5)
    for s in (0, 7):
        v = torch.tensor(rng.standard_normal(N), device="cuda")
        gg, yy, ll = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
        h = 1e-6
        Jp = iga.iga_reduced_gradient(ctx, M, K, load, work.beta, (u[s] + h * v).contiguous(), gg,
                                      yy, ll, 1e-12)[0]
        Jm = iga.iga_reduced_gradient(ctx, M, K, load, work.beta, (u[s] - h * v).contiguous(), gg,
                                      yy, ll, 1e-12)[0]
        fd = (Jp - Jm) / (2 * h)
        an = float(torch.dot(g[s], v))
        assert abs(fd - an) < 1e-5 * max(1e-6, abs(an)), (s, fd, an)
    # the adjoint satisfies K lam = b - M y to the solve tolerance
    s = 3
    Ky = torch.empty(N, dtype=torch.float64, device="cuda")
    iga.iga_kron_apply(ctx, K, 1.0, lam[s].contiguous(), 0.0, Ky)
    My = torch.empty(N, dtype=torch.float64, device="cuda")
    iga.iga_kron_apply(ctx, M, 1.0, y[s].contiguous(), 0.0, My)
    bfull = torch.empty(tuple(n), dtype=torch.float64, device="cuda")
    load.full(ctx, bfull)
    r = Ky - (bfull.reshape(-1) - My)
    assert float(r.norm() / (bfull.norm() + My.norm())) < 1e-10
