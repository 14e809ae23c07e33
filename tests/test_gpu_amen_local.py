"""GPU parity of the block-AMEn solve without full-size operator applies
(IGA_RESID_LOCAL: projected residuals as the stopping test, Khatri-Rao
sketches of the residual for the enrichment) against the oracle's direct
sparse solve of the 3-D assembled system on small grids, including TT-matrix
operators of rank > 1 (random cubic volume) whose univariate factors are not
symmetric; at the full 64-element quarter annulus against the oracle's
reduced-system solve; and the TT output against the full-vector output."""
import math

import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.kkt import kkt_residual, kkt_solve
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _oracle_system(work):
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, b = assemble_band(work.geometry, disc, work.target)
    return band_to_csr(Mb, True), band_to_csr(Kb, True), b[1:-1, 1:-1, 1:-1].ravel()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    ("annulus", wl.small(wl.quarter_annulus(), 3, 7,
                         wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-4, tol=1e-12)),
    ("twisted", wl.small(wl.quarter_annulus(twist=math.pi / 4), 2, 9,
                         wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-3, tol=1e-12)),
    ("random", wl.small(wl.random_volume(), 2, 6, wl.Target(wl.TARGET_SINPROD), beta=1e-4,
                        tol=1e-12)),
    ("random_e10", wl.small(wl.random_volume(), 2, 10, wl.Target(wl.TARGET_SINPROD), beta=1e-6,
                            tol=1e-12)),
]


@pytest.mark.parametrize("name,work", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("trunc", [0, 1], ids=["pivoted", "svd"])
def test_local_mode_matches_direct(env, name, work, prec, trunc):
    ctx, torch, iga = env
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    info = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, y, u, lam, tol=1e-10,
                                  precision=prec, truncation=trunc,
                                  residual=iga.IGA_RESID_LOCAL, max_sweeps=12)
    assert info["converged"], info
    assert info["refinements"] == 0
    Mo, Ko, b = _oracle_system(work)
    y, u, lam = (t.cpu().numpy() for t in (y, u, lam))
    # the projected residual bounds the true one from below only: the true
    # residual, measured with the oracle's 3-D matrices, within 100 x tol
    assert kkt_residual(Mo, Ko, work.beta, b, y, u, lam) < 1e-8
    yo, uo, lo = kkt_solve(Mo, Ko, work.beta, b)
    for got, ref in ((y, yo), (u, uo), (lam, lo)):
        assert _rel(got, ref) < 1e-6, (name, _rel(got, ref))


def test_local_mode_tt_output_expands_to_the_full_solution(env):
    ctx, torch, iga = env
    work = CASES[2][1]
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    ni = M.info()["n"]
    N = int(np.prod(ni))
    opts = dict(tol=1e-10, residual=iga.IGA_RESID_LOCAL, max_sweeps=12)
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    info = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, y, u, lam, **opts)
    assert info["converged"]
    ty, tu, tl, info2 = iga.iga_kkt_solve_amen_tt(ctx, M, K, load, work.beta, **opts)
    assert info2["converged"] and info2["sweeps"] == info["sweeps"]
    for t, full in ((ty, y), (tu, u), (tl, lam)):
        out = torch.empty(ni, dtype=torch.float64, device="cuda")
        t.full(ctx, out)
        # same seeds and moves; only the order of atomic FP64 sums may differ
        assert float((out.reshape(-1) - full).norm() / full.norm()) < 1e-9
        # the TT ranks are those of the block TT
        _, ranks = t.info()
        assert max(ranks) <= info["max_rank"]


def test_local_mode_zero_load_gives_zero_tts(env):
    ctx, torch, iga = env
    work = CASES[0][1]
    M, K, _ = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    ni = M.info()["n"]
    ty, tu, tl, info = iga.iga_kkt_solve_amen_tt(ctx, M, K, None, work.beta,
                                                 residual=iga.IGA_RESID_LOCAL)
    assert info["converged"]
    for t in (ty, tu, tl):
        out = torch.ones(ni, dtype=torch.float64, device="cuda")
        t.full(ctx, out)
        assert float(out.abs().max()) == 0.0


def test_local_mode_rejects_wide_kick(env):
    ctx, torch, iga = env
    work = CASES[0][1]
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    with pytest.raises(iga.IgaError):
        iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, y, u, lam,
                               residual=iga.IGA_RESID_LOCAL, kick_rank=17)


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_local_mode_config2_matches_oracle(env, prec):
    """The 64-element quarter annulus (weights interpolated, TT tolerance
    1e-10 on both sides) solved without any full-size operator apply to a
    projected residual of 1e-9: the true residual (the library's FP64 KKT
    apply) and y, u, lambda against the oracle's reduced-system solve."""
    from oracle.solve import interior_operators_interp, solve_kkt
    ctx, torch, iga = env
    work = wl.config(2)
    Mt, Kt, diag, bo = interior_operators_interp(work.space, work.geometry, work.target, 1e-10)
    yo, uo, lo, _ = solve_kkt(Mt, Kt, diag, bo, work.beta, tol=1e-12)
    M, K, load = iga.iga_lowrank_assemble_interp(ctx, work.geometry, work.space, work.target,
                                                 1e-10)
    ni = M.info()["n"]
    N = int(np.prod(ni))
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    info = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, y, u, lam, tol=1e-9,
                                  precision=prec, residual=iga.IGA_RESID_LOCAL, max_sweeps=12)
    assert info["converged"], info
    z = torch.cat([y, u, lam])
    out = torch.empty_like(z)
    iga.iga_kkt_apply(ctx, M, K, work.beta, z, out)
    bfull = torch.empty(ni, dtype=torch.float64, device="cuda")
    load.full(ctx, bfull)
    b = torch.zeros_like(z)
    b[:N] = bfull.reshape(-1)
    assert float((b - out).norm() / b.norm()) <= 1e-7
    for g, ref, name in ((y, yo, "y"), (u, uo, "u"), (lam, lo, "lam")):
        err = np.linalg.norm(g.cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err <= 1e-6, (name, err)


def test_residual_rows_match_the_full_residual(env):
    """iga_kkt_residual_rows (operator entries from the bands, solution values
    from the TT cores, nothing of full size) against the full FP64 KKT
    residual of the expanded solution, row by row, including rows on the
    boundary layer of the interior grid."""
    ctx, torch, iga = env
    work = CASES[3][1]
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    ni = M.info()["n"]
    N = int(np.prod(ni))
    ty, tu, tl, info = iga.iga_kkt_solve_amen_tt(ctx, M, K, load, work.beta, tol=1e-4,
                                                 residual=iga.IGA_RESID_LOCAL)
    z = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    for f, t in enumerate((ty, tu, tl)):
        t.full(ctx, z[f * N:(f + 1) * N].view(ni))
    out = torch.empty_like(z)
    iga.iga_kkt_apply(ctx, M, K, work.beta, z, out)
    bfull = torch.empty(ni, dtype=torch.float64, device="cuda")
    load.full(ctx, bfull)
    b = torch.zeros_like(z)
    b[:N] = bfull.reshape(-1)
    res = (b - out).cpu().numpy().reshape(3, *ni)
    rng = np.random.default_rng(7)
    rows = np.stack([rng.integers(0, ni[d], 40) for d in range(3)], axis=1)
    rows[0] = (0, 0, 0)
    rows[1] = tuple(x - 1 for x in ni)
    got = iga.iga_kkt_residual_rows(ctx, M, K, work.beta, load, ty, tu, tl, rows)
    ref = np.stack([res[e][tuple(rows.T)] for e in range(3)], axis=1)
    scale = float(b.norm())
    assert np.abs(got - ref).max() <= 1e-12 * scale, np.abs(got - ref).max() / scale
    # the residual is not negligible at this tolerance, so the comparison is not vacuous
    assert np.abs(ref).max() > 1e-9 * scale
    with pytest.raises(iga.IgaError):
        iga.iga_kkt_residual_rows(ctx, M, K, work.beta, load, ty, tu, tl, [[ni[0], 0, 0]])


@pytest.mark.parametrize("name,work", CASES[2:], ids=[c[0] for c in CASES[2:]])
@pytest.mark.parametrize("resid", [0, 1], ids=["full", "local"])
def test_tf32_solve_with_tensor_core_band_contraction(env, name, work, resid):
    """IGA_TF32 on the random volume: the middle core's banded contraction of
    the TT-matrix operators (blocks of TT ranks >= 4) runs as batched TF32
    GEMMs on the tensor cores, the local systems are refined in FP64, and the
    solution must match the oracle's direct solve as in the FP64 path."""
    ctx, torch, iga = env
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    assert max(min(M.block_ranks(k)) for k in range(M.info()["nblocks"])) >= 4
    N = int(np.prod(M.info()["n"]))
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    ctx.profile_begin("tc_gemm_tf32_kernel")
    info = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, y, u, lam, tol=1e-10,
                                  precision=iga.IGA_TF32, residual=resid, max_sweeps=12)
    prof = ctx.profile_end()
    assert info["converged"], info
    assert prof["launches"] > 0          # the tensor-core path ran
    Mo, Ko, b = _oracle_system(work)
    y, u, lam = (t.cpu().numpy() for t in (y, u, lam))
    assert kkt_residual(Mo, Ko, work.beta, b, y, u, lam) < 1e-8
    yo, uo, lo = kkt_solve(Mo, Ko, work.beta, b)
    for got, ref in ((y, yo), (u, uo), (lam, lo)):
        assert _rel(got, ref) < 1e-6, (name, _rel(got, ref))


@pytest.mark.parametrize("trunc", [0, 1], ids=["pivoted", "svd"])
def test_state_weight_keeps_the_solution(env, trunc):
    """A weighted state in the truncation (state_weight) changes the ranks the
    solve keeps, never the solution it converges to."""
    ctx, torch, iga = env
    work = CASES[3][1]
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    N = int(np.prod(M.info()["n"]))
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    info = iga.iga_kkt_solve_amen(ctx, M, K, load, work.beta, y, u, lam, tol=1e-10,
                                  truncation=trunc, residual=iga.IGA_RESID_LOCAL,
                                  max_sweeps=12, state_weight=1e3)
    assert info["converged"], info
    Mo, Ko, b = _oracle_system(work)
    yo, uo, lo = kkt_solve(Mo, Ko, work.beta, b)
    for got, ref in ((y, yo), (u, uo), (lam, lo)):
        assert _rel(got.cpu().numpy(), ref) < 1e-6
