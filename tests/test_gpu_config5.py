"""Full-size random cubic volume (degree 2, 512 elements per direction, TT tolerance
1e-8): weight ranks, sampled-row parity of the assembled operators, and the TF32
tensor-core TT-matrix apply at sampled rows."""
import numpy as np
import pytest

from oracle.assemble import Discretisation, sampled_rows
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch

pytestmark = pytest.mark.gpu


def test_config5_assembly_and_tf32_apply():
    ctx, torch, iga = ctx_and_torch()
    work = wl.config(5)
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    assert min(M.block_ranks(0)) > 20                  # a genuinely high-rank geometry
    assert load is not None
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    n = disc.n
    rng = np.random.default_rng(55)
    rows = np.stack([rng.integers(1, n[d] - 1, 3) for d in range(3)], axis=1)
    Mr, Kr = sampled_rows(work.geometry, disc, rows)
    p = 2
    ni = M.info()["n"]
    N = int(np.prod(ni))
    x = torch.randn(N, dtype=torch.float32, device="cuda")
    xh = x.double().cpu().numpy().reshape(ni)
    y = torch.empty_like(x)
    for op, ref in ((M, Mr), (K, Kr)):
        # operator rows from the device factors (TT-matrix terms summed)
        got_rows = []
        for s, r in enumerate(rows):
            ii = r - 1
            acc = np.zeros((5, 5, 5))
            for k in range(op.info()["nblocks"]):
                R1, R2 = op.block_ranks(k)
                b0, b1, b2 = (op.bands(ctx, k, d) for d in range(3))
                acc += np.einsum("ai,abj,bk->ijk", b0[:, ii[0]], b1[:, :, ii[1]], b2[:, ii[2]])
            want = ref[s].copy()
            for d in range(3):
                for o in range(5):
                    j = r[d] + o - p
                    if j < 1 or j > n[d] - 2:
                        idx = [slice(None)] * 3
                        idx[d] = o
                        want[tuple(idx)] = 0.0
            assert np.linalg.norm(acc - want) < 1e-6 * np.linalg.norm(want), (s, r)
            got_rows.append(want)
        # TF32 apply against the oracle rows times x
        iga.iga_kron_apply(ctx, op, 1.0, x, 0.0, y, tf32=True)
        yh = y.double().cpu().numpy().reshape(ni)
        for s, r in enumerate(rows):
            ii = r - 1
            sl = tuple(slice(ii[d] - p, ii[d] + p + 1) for d in range(3))
            pad = np.zeros((5, 5, 5))
            lo = [max(0, ii[d] - p) for d in range(3)]
            hi = [min(ni[d], ii[d] + p + 1) for d in range(3)]
            sub = xh[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]]
            off = [lo[d] - (ii[d] - p) for d in range(3)]
            pad[off[0]:off[0] + sub.shape[0], off[1]:off[1] + sub.shape[1],
                off[2]:off[2] + sub.shape[2]] = sub
            want = float(np.sum(got_rows[s] * pad))
            scale = float(np.sum(np.abs(got_rows[s]) * np.abs(pad)))
            assert abs(yh[tuple(ii)] - want) < 1e-3 * scale, (s, yh[tuple(ii)], want)


def _tt_values(cores, pts):
    """Values of a TT (numpy cores (1,n1,r1), (r1,n2,r2), (r2,n3,1)) at the
    interior multi-indices pts (S, 3)."""
    c0, c1, c2 = cores
    return np.einsum("sa,asb,bs->s", c0[0, pts[:, 0], :], c1[:, pts[:, 1], :], c2[:, pts[:, 2], 0])


def test_config5_solve_without_full_applies():
    """The random-volume KKT solve (1.34e8 unknowns per field) in mixed
    precision without any full-size operator apply (IGA_RESID_LOCAL, solution
    as the block TT), three sweeps.  Its residual is measured at 128 uniformly
    sampled rows of all three KKT equations twice: with the library's row
    evaluation of the low-rank operators (iga_kkt_residual_rows), and with the
    oracle's exact row integrals of M and K (`sampled_rows`) and load entries
    (`sampled_load`) applied to the TT solution.  The two estimates of the
    relative residual, sqrt(N / S sum of squares) / ||b||, must agree (the
    operators differ by the TT truncation at 1e-8 and the weight
    interpolation); and the solve must have reduced the residual well below
    that of the zero iterate (1)."""
    from oracle.assemble import sampled_load
    ctx, torch, iga = ctx_and_torch()
    work = wl.config(5)
    M, K, load = iga.iga_lowrank_assemble_interp(ctx, work.geometry, work.space, work.target,
                                                 work.tol)
    ni = M.info()["n"]
    N = int(np.prod(ni))
    ty, tu, tl, info = iga.iga_kkt_solve_amen_tt(ctx, M, K, load, work.beta, tol=1e-6,
                                                 precision=iga.IGA_FP32, trunc_tol=1e-6,
                                                 residual=iga.IGA_RESID_LOCAL, max_sweeps=3)
    assert info["sweeps"] == 3 and info["max_rank"] > 4
    bfull = torch.empty(ni, dtype=torch.float64, device="cuda")
    load.full(ctx, bfull)
    bnorm = float(bfull.norm())
    del bfull
    rng = np.random.default_rng(505)
    S = 128
    rows = np.stack([rng.integers(0, ni[d], S) for d in range(3)], axis=1)
    got = iga.iga_kkt_residual_rows(ctx, M, K, work.beta, load, ty, tu, tl, rows)
    est_lib = np.sqrt(N / S * np.sum(got ** 2)) / bnorm
    # the oracle's exact rows (full-grid indices = interior + 1)
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    n = disc.n
    full_rows = rows + 1
    Mr, Kr = sampled_rows(work.geometry, disc, full_rows)
    br = sampled_load(work.geometry, disc, work.target, full_rows)
    cores = [t.cores(ctx) for t in (ty, tu, tl)]
    p = 2
    res = np.zeros((S, 3))
    offs = np.array([(a, b, c) for a in range(5) for b in range(5) for c in range(5)])
    for s, r in enumerate(full_rows):
        j = r[None, :] + offs - p                       # full-grid stencil indices
        ok = np.all((j >= 1) & (j <= np.array(n) - 2), axis=1)
        jj = j[ok] - 1
        zy, zu, zl = (_tt_values(c, jj) for c in cores)
        m = Mr[s][tuple(offs[ok].T)]
        k = Kr[s][tuple(offs[ok].T)]
        res[s, 0] = br[s] - m @ zy - k @ zl
        res[s, 1] = -(work.beta * (m @ zu) - m @ zl)
        res[s, 2] = -(k @ zy - m @ zu)
    est_oracle = np.sqrt(N / S * np.sum(res ** 2)) / bnorm
    assert est_oracle < 0.2, est_oracle
    assert abs(est_lib - est_oracle) <= 0.1 * est_oracle, (est_lib, est_oracle)
    # row by row, the two evaluations agree to the operators' difference
    scale = np.abs(res).max()
    assert np.abs(got - res).max() <= 0.1 * scale, (np.abs(got - res).max(), scale)
