"""GPU parity of steps a1-a4 (sampling, TT-SVD, univariate assembly) against the oracle."""
import math

import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr, sample_weights, sampled_rows
from oracle.lowrank import kron_matrix, tt_full, tt_ranks, univariate_band, tt_svd
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch, fro_rel, op_terms

pytestmark = pytest.mark.gpu

GEOS = {
    "cube": wl.unit_cube(),
    "annulus": wl.quarter_annulus(),
    "twisted": wl.quarter_annulus(twist=math.pi / 4),
    "random": wl.random_volume(),
}


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _disc(space):
    return Discretisation(space.degree, space.knots, space.nquad)


@pytest.mark.parametrize("name", ["annulus", "twisted", "random"])
def test_sample_weights(env, name):
    ctx, torch, iga = env
    space = wl.uniform_space(3, 5)
    disc = _disc(space)
    tgt = wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1)
    Q = [e * space.nquad for e in disc.E]
    out = torch.empty((8, *Q), dtype=torch.float64, device="cuda")
    iga.iga_sample_weights(ctx, GEOS[name], space, tgt, out)
    G, om, Qm, _ = sample_weights(GEOS[name], disc)
    _, gs = disc.gauss_grid()
    g = np.einsum("a,b,c->abc", *gs)
    from oracle.assemble import evaluate_target
    yh = evaluate_target(tgt, G.reshape(-1, 3)).reshape(om.shape)
    ref = [om * g, Qm[..., 0, 0] * g, Qm[..., 0, 1] * g, Qm[..., 0, 2] * g, Qm[..., 1, 1] * g,
           Qm[..., 1, 2] * g, Qm[..., 2, 2] * g, yh * om * g]
    got = out.cpu().numpy()
    scale = max(np.abs(r).max() for r in ref[1:7])
    for c in range(8):
        s = scale if 1 <= c <= 6 else np.abs(ref[c]).max()
        assert np.abs(got[c] - ref[c]).max() < 1e-13 * s, c


@pytest.mark.parametrize("interior", [0, 1])
@pytest.mark.parametrize("deriv", [(0, 0), (1, 1), (1, 0), (0, 1)])
def test_univariate_bands(env, interior, deriv):
    ctx, torch, iga = env
    knots = np.array([0, 0, 0, 0, 0.1, 0.3, 0.3, 0.55, 0.8, 1, 1, 1, 1.0])   # ragged, repeated
    space = wl.Space((3, 3, 3), (knots, knots, knots), 4)
    disc = _disc(space)
    E, q, n = disc.E[0], space.nquad, disc.n[0]
    T = 5
    w = np.random.default_rng(1).standard_normal((T, E * q))
    wt = torch.tensor(w, device="cuda")
    nrow = n - 2 * interior
    band = torch.empty((T, nrow, 7), dtype=torch.float64, device="cuda")
    iga.iga_assemble_bands(ctx, space, 0, wt, deriv[0], deriv[1], interior, band)
    got = band.cpu().numpy()
    for t in range(T):
        ref = univariate_band(disc.V[0], disc.D[0], disc.first[0], n, w[t].reshape(E, q), *deriv)
        if interior:
            ref = ref[1:-1].copy()
            for i in range(nrow):             # drop couplings to the boundary functions
                for o in range(7):
                    j = i + 1 + o - 3
                    if j < 1 or j > n - 2:
                        ref[i, o] = 0.0
        assert np.abs(got[t] - ref).max() < 1e-13 * np.abs(ref).max()


def _random_tt(n, r, seed):
    rng = np.random.default_rng(seed)
    ranks = (1,) + tuple(r) + (1,)
    return [rng.standard_normal((ranks[d], n[d], ranks[d + 1])) for d in range(3)]


@pytest.mark.parametrize("n,r", [((30, 41, 23), (3, 5)), ((64, 16, 80), (1, 1)), ((17, 9, 40), (9, 12))])
def test_tt_svd_exact_rank(env, n, r):
    ctx, torch, iga = env
    W = tt_full(_random_tt(n, r, 3))
    tt = iga.iga_tt_svd(ctx, torch.tensor(W, device="cuda"), 1e-12)
    (nn, rr) = tt.info()
    assert nn == n and rr == r
    full = torch.empty(n, dtype=torch.float64, device="cuda")
    tt.full(ctx, full)
    assert np.linalg.norm(full.cpu().numpy() - W) < 1e-12 * np.linalg.norm(W)
    # host copies of the cores multiply out to the same tensor
    assert np.linalg.norm(tt_full(tt.cores(ctx)) - W) < 1e-12 * np.linalg.norm(W)


@pytest.mark.parametrize("tol", [1e-2, 1e-4])
def test_tt_svd_error_bound(env, tol):
    ctx, torch, iga = env
    rng = np.random.default_rng(5)
    # smooth tensor with decaying spectrum plus noise
    x = np.linspace(0, 1, 24)
    W = np.exp(-np.add.outer(np.add.outer(x, 2 * x), x) ** 2) + 1e-3 * rng.standard_normal((24, 24, 24))
    tt = iga.iga_tt_svd(ctx, torch.tensor(W, device="cuda"), tol)
    err = np.linalg.norm(tt_full(tt.cores(ctx)) - W) / np.linalg.norm(W)
    assert err <= tol * 1.0001
    ref = tt_svd(W, tol)
    # the sketched ranks may exceed the exact truncation ranks by a little, never fall short
    assert all(a >= b for a, b in zip(tt.info()[1], tt_ranks(ref)))


def test_tt_svd_zero_is_rank_zero(env):
    ctx, torch, iga = env
    assert iga.iga_tt_svd(ctx, torch.zeros((4, 5, 6), dtype=torch.float64, device="cuda"), 1e-8) is None


CASES = [("cube", 2, 4, 1e-12, 1e-12), ("annulus", 3, 5, 1e-12, 1e-11),
         ("twisted", 2, 6, 1e-12, 1e-11), ("random", 2, 4, 1e-6, 1e-5)]


@pytest.mark.parametrize("name,p,E,tol,bar", CASES)
def test_lowrank_assemble_matches_3d_assembly(env, name, p, E, tol, bar):
    ctx, torch, iga = env
    geo = GEOS[name]
    tgt = wl.Target(wl.TARGET_SINPROD) if name in ("cube", "random") else wl.Target(
        wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1)
    space = wl.uniform_space(p, E)
    M, K, load = iga.iga_lowrank_assemble(ctx, geo, space, tgt, tol)
    disc = _disc(space)
    Mb, Kb, b = assemble_band(geo, disc, tgt)
    Mo, Ko = band_to_csr(Mb, interior=True), band_to_csr(Kb, interior=True)
    assert fro_rel(kron_matrix(op_terms(ctx, M)), Mo) < bar
    assert fro_rel(kron_matrix(op_terms(ctx, K)), Ko) < bar
    bl = tt_full(load.cores(ctx))
    bo = b[1:-1, 1:-1, 1:-1]
    assert np.linalg.norm(bl - bo) < bar * np.linalg.norm(bo)


def test_config2_sampled_rows(env):
    """Full-size quarter annulus (degree 3, 64 elements): sampled rows against the definition."""
    ctx, torch, iga = env
    work = wl.config(2)
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    disc = _disc(work.space)
    rng = np.random.default_rng(7)
    n = disc.n
    rows = np.stack([rng.integers(1, n[d] - 1, 6) for d in range(3)], axis=1)
    rows[0] = (1, 1, 1)
    rows[1] = (n[0] - 2, n[1] - 2, n[2] - 2)
    Mr, Kr = sampled_rows(work.geometry, disc, rows)
    p = 3
    for op, ref in ((M, Mr), (K, Kr)):
        terms = []
        for k in range(op.info()["nblocks"]):
            terms.append([op.bands(ctx, k, d)[0] if d != 1 else op.bands(ctx, k, 1)[0, 0]
                          for d in range(3)])
        for s, r in enumerate(rows):
            got = np.zeros((7, 7, 7))
            ii = r - 1                                      # interior index
            for t in terms:
                got += np.einsum("a,b,c->abc", t[0][ii[0]], t[1][ii[1]], t[2][ii[2]])
            want = ref[s].copy()
            # interior operator: couplings to boundary functions are omitted
            for d in range(3):
                for o in range(7):
                    j = r[d] + o - p
                    if j < 1 or j > n[d] - 2:
                        idx = [slice(None)] * 3
                        idx[d] = o
                        want[tuple(idx)] = 0.0
            assert np.linalg.norm(got - want) < 1e-11 * np.linalg.norm(want), (s, r)


@pytest.mark.parametrize("scale,rank_one", [(0.2, True), (5.0, False)])
def test_tt_svd_rank_one_cross(env, scale, rank_one):
    """Rank-1 tensor plus noise of norm scale * tol * |W|: the cross test accepts only
    below the per-unfolding threshold, otherwise the sketch runs; the bound holds in both."""
    ctx, torch, iga = env
    tol = 1e-4
    W0 = tt_full(_random_tt((40, 33, 57), (1, 1), 11))
    noise = np.random.default_rng(12).standard_normal(W0.shape)
    W = W0 + scale * tol * np.linalg.norm(W0) * noise / np.linalg.norm(noise)
    tt = iga.iga_tt_svd(ctx, torch.tensor(W, device="cuda"), tol)
    err = np.linalg.norm(tt_full(tt.cores(ctx)) - W) / np.linalg.norm(W)
    assert err <= tol * 1.0001
    if rank_one:
        assert tt.info()[1] == (1, 1)
    else:
        assert all(a >= b for a, b in zip(tt.info()[1], tt_ranks(tt_svd(W, tol))))
        assert max(tt.info()[1]) > 1
