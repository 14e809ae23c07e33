"""GPU parity of the parabolic KKT solve (Sec. 4 eqs. timeDiscrete and
KKTSystem; block AMEn on the space-time TT, Sec. 5) against the oracle's
direct solve of the assembled space-time system, element by element.

Both sides take the same desired-state load: the spatial load vector of the
target (each side its own assembly) times a time profile, b_k = tau g(t_k) b."""
import math

import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.parabolic import kkt_residual_parabolic, kkt_solve_parabolic
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _profile(nt, tau):
    t = tau * np.arange(1, nt + 1)
    return 0.5 + np.sin(math.pi * t)


def _oracle(work, nt, tau):
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, b = assemble_band(work.geometry, disc, work.target)
    M, K = band_to_csr(Mb, True), band_to_csr(Kb, True)
    b = b[1:-1, 1:-1, 1:-1].ravel()
    B = tau * _profile(nt, tau)[:, None] * b[None, :]
    return M, K, B


def _solve(env, work, nt, tau, zero_load=False, **opts):
    ctx, torch, iga = env
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    load.full(ctx, b)
    g = torch.tensor(tau * _profile(nt, tau), dtype=torch.float64, device="cuda")
    B = (g[:, None] * b[None, :]).contiguous()
    if zero_load:
        B.zero_()
    y, u, lam = (torch.empty((nt, N), dtype=torch.float64, device="cuda") for _ in range(3))
    info = iga.iga_kkt_solve_parabolic(ctx, M, K, nt, tau, B, work.beta, y, u, lam, **opts)
    return info, y.cpu().numpy(), u.cpu().numpy(), lam.cpu().numpy()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    ("cube_nt4", wl.small(wl.unit_cube(), 2, 5, beta=1e-2, tol=1e-12), 4, 0.25),
    ("annulus_nt6", wl.small(wl.quarter_annulus(), 3, 5,
                             wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-4,
                             tol=1e-12), 6, 1.0 / 6),
    ("twisted_nt10", wl.small(wl.quarter_annulus(twist=math.pi / 4), 2, 6,
                              wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-3,
                              tol=1e-12), 10, 0.1),
    # TT-matrix operators with weight ranks > 1 (random cubic volume)
    ("random_nt3", wl.small(wl.random_volume(), 2, 5, wl.Target(wl.TARGET_SINPROD), beta=1e-4,
                            tol=1e-12), 3, 0.2),
    # one step: the stationary layout with K + M / tau
    ("annulus_nt1", wl.small(wl.quarter_annulus(), 2, 6,
                             wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-3,
                             tol=1e-12), 1, 0.5),
]


@pytest.mark.parametrize("name,work,nt,tau", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_parabolic_solve_matches_direct(env, name, work, nt, tau, prec):
    info, y, u, lam = _solve(env, work, nt, tau, tol=1e-10, precision=prec)
    assert info["converged"], info
    M, K, B = _oracle(work, nt, tau)
    # the GPU solution's residual in the oracle's assembled space-time system
    assert kkt_residual_parabolic(M, K, tau, work.beta, B, y, u, lam) < 1e-9
    yo, uo, lo = kkt_solve_parabolic(M, K, tau, work.beta, B)
    for got, ref in ((y, yo), (u, uo), (lam, lo)):
        assert _rel(got, ref) < 1e-6, (name, _rel(got, ref))


def test_parabolic_solve_with_svd_moves(env):
    name, work, nt, tau = CASES[1]
    info, y, u, lam = _solve(env, work, nt, tau, tol=1e-10, truncation=1)
    assert info["converged"], info
    M, K, B = _oracle(work, nt, tau)
    yo, uo, lo = kkt_solve_parabolic(M, K, tau, work.beta, B)
    for got, ref in ((y, yo), (u, uo), (lam, lo)):
        assert _rel(got, ref) < 1e-6


def test_parabolic_zero_load_gives_zero(env):
    name, work, nt, tau = CASES[0]
    info, y, u, lam = _solve(env, work, nt, tau, zero_load=True)
    assert info["converged"]
    assert not y.any() and not u.any() and not lam.any()


def test_parabolic_rejects_bad_arguments(env):
    ctx, torch, iga = env
    work = CASES[0][1]
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    t = [torch.zeros((2, N), dtype=torch.float64, device="cuda") for _ in range(4)]
    for nt, tau, beta, kw in ((0, 0.5, 1e-2, {}), (2, 0.0, 1e-2, {}), (2, 0.5, 0.0, {}),
                              (2, 0.5, 1e-2, {"residual": 1})):
        B = t[0] if nt == 2 else None
        with pytest.raises(iga.IgaError):
            iga.iga_kkt_solve_parabolic(ctx, M, K, nt, tau, B, beta, t[1], t[2], t[3], **kw)
    with pytest.raises(iga.IgaError):
        # wrong element count
        iga.iga_kkt_solve_parabolic(ctx, M, K, 3, 0.5, t[0], 1e-2, t[1], t[2], t[3])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_parabolic_bench_workload_rows(env, prec):
    """The bench's parabolic case at full size: the quarter annulus of degree 3
    with 64 elements per direction (interpolated weights), 10 steps of size
    0.1, b_k = tau (1/2 + sin(pi t_k)) b.  Sampled rows of the three
    equations, every step, evaluated with the oracle's own row integrals of
    M and K and load entries applied to the GPU solution; a row's residual
    never exceeds the residual's 2-norm."""
    from oracle.assemble import sampled_load, sampled_rows
    from test_gpu_config2 import _apply_row
    ctx, torch, iga = env
    work = wl.config(2)
    nt, tau = 10, 0.1
    M, K, load = iga.iga_lowrank_assemble_interp(ctx, work.geometry, work.space, work.target,
                                                 work.tol)
    ni = M.info()["n"]
    N = int(np.prod(ni))
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    load.full(ctx, b)
    g = tau * _profile(nt, tau)
    B = (torch.tensor(g, dtype=torch.float64, device="cuda")[:, None] * b[None, :]).contiguous()
    y, u, lam = (torch.empty((nt, N), dtype=torch.float64, device="cuda") for _ in range(3))
    info = iga.iga_kkt_solve_parabolic(ctx, M, K, nt, tau, B, work.beta, y, u, lam, tol=1e-6,
                                       precision=prec)
    assert info["converged"] and info["residual"] <= 1e-6, info
    Fn = float(B.norm())
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    n = disc.n
    rng = np.random.default_rng(1010)
    rows = np.stack([rng.integers(1, n[d] - 1, 6) for d in range(3)], axis=1)
    rows[0] = (1, 1, 1)
    Mr, Kr = sampled_rows(work.geometry, disc, rows)
    br = sampled_load(work.geometry, disc, work.target, rows)
    Y, U, L = (t.cpu().numpy().reshape((nt,) + tuple(ni)) for t in (y, u, lam))
    bound = (1e-6 + 10 * work.tol) * Fn
    for s, r in enumerate(rows):
        my = [_apply_row(Mr[s], Y[k], r, n) for k in range(nt)]
        ml = [_apply_row(Mr[s], L[k], r, n) for k in range(nt)]
        for k in range(nt):
            ky, kl = _apply_row(Kr[s], Y[k], r, n), _apply_row(Kr[s], L[k], r, n)
            mu = _apply_row(Mr[s], U[k], r, n)
            ry = tau * (my[k] + kl) + ml[k] - (ml[k + 1] if k + 1 < nt else 0.0) - g[k] * br[s]
            ru = tau * (work.beta * mu - ml[k])
            rl = tau * (ky - mu) + my[k] - (my[k - 1] if k > 0 else 0.0)
            for e, v in enumerate((ry, ru, rl)):
                assert abs(v) <= bound, (s, r, k, e, v, bound)


@pytest.mark.parametrize("nt", [2, 24])
def test_parabolic_tf32_and_longer_horizons(env, nt):
    """IGA_TF32 (interface products on the tensor cores once they are large,
    FP64 refinement) and horizons of 2 and 24 steps against the direct
    solve."""
    work = CASES[0][1]
    tau = 1.0 / nt
    info, y, u, lam = _solve(env, work, nt, tau, tol=1e-10, precision=2)
    assert info["converged"], info
    M, K, B = _oracle(work, nt, tau)
    yo, uo, lo = kkt_solve_parabolic(M, K, tau, work.beta, B)
    for got, ref in ((y, yo), (u, uo), (lam, lo)):
        assert _rel(got, ref) < 1e-6
