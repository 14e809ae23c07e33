"""Full-size twisted quarter annulus (degree 3, 256 elements per direction):
sampled-row parity of the operators and the load, and the KKT solve to a
relative residual of 1e-6 for beta in {1e-2, 1e-4, 1e-6}."""
import numpy as np
import pytest

from oracle.assemble import Discretisation, sampled_load, sampled_rows
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    ctx, torch, iga = ctx_and_torch()
    work = wl.config(3)
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    return ctx, torch, iga, work, M, K, load


def _rows(n, k, seed):
    rng = np.random.default_rng(seed)
    rows = np.stack([rng.integers(1, n[d] - 1, k) for d in range(3)], axis=1)
    rows[0] = (1, 1, 1)
    rows[-1] = tuple(x - 2 for x in n)
    return rows


def test_config3_operators_and_load_at_sampled_rows(setup):
    ctx, torch, iga, work, M, K, load = setup
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    n = disc.n
    rows = _rows(n, 4, 31)
    Mr, Kr = sampled_rows(work.geometry, disc, rows)
    br = sampled_load(work.geometry, disc, work.target, rows)
    ni = M.info()["n"]
    bfull = torch.empty(ni, dtype=torch.float64, device="cuda")
    load.full(ctx, bfull)
    bh = bfull.cpu().numpy()
    # the load density is TT-truncated at tol = 1e-8 (it is not rank 1 on this
    # geometry): every entry is within 10 tol of the Frobenius norm of b
    bnorm = float(np.linalg.norm(bh))
    for s, r in enumerate(rows):
        assert abs(bh[tuple(r - 1)] - br[s]) < 10 * work.tol * bnorm
    p = 3
    for op, ref in ((M, Mr), (K, Kr)):
        terms = [[op.bands(ctx, k, d)[0] if d != 1 else op.bands(ctx, k, 1)[0, 0] for d in range(3)]
                 for k in range(op.info()["nblocks"])]
        for s, r in enumerate(rows):
            got = np.zeros((7, 7, 7))
            ii = r - 1
            for t in terms:
                got += np.einsum("a,b,c->abc", t[0][ii[0]], t[1][ii[1]], t[2][ii[2]])
            want = ref[s].copy()
            for d in range(3):
                for o in range(7):
                    j = r[d] + o - p
                    if j < 1 or j > n[d] - 2:
                        idx = [slice(None)] * 3
                        idx[d] = o
                        want[tuple(idx)] = 0.0
            # weights are TT-truncated at 1e-8: the factors agree to 10x that
            assert np.linalg.norm(got - want) < 1e-7 * np.linalg.norm(want)


@pytest.mark.parametrize("beta,prec", [(1e-2, 0), (1e-4, 0), (1e-6, 0), (1e-4, 2), (1e-6, 2)],
                         ids=["1e-2", "1e-4", "1e-6", "1e-4-tf32", "1e-6-tf32"])
def test_config3_kkt_solve(setup, beta, prec):
    """FP64 solves, and solves whose large local interface products run on the
    tensor cores in TF32 (IGA_TF32) inside the FP64 refinement."""
    ctx, torch, iga, work, M, K, load = setup
    N = int(np.prod(M.info()["n"]))
    y, u, lam = (torch.empty(N, dtype=torch.float64, device="cuda") for _ in range(3))
    if prec == 2:
        ctx.profile_begin("tc_gemm_tf32_kernel")
    info = iga.iga_kkt_solve_amen(ctx, M, K, load, beta, y, u, lam, tol=1e-6, precision=prec)
    if prec == 2:
        assert ctx.profile_end()["launches"] > 0          # the tensor-core products ran
    assert info["converged"], info
    # independent residual check with the (row-verified) operator apply
    z = torch.cat([y, u, lam])
    out = torch.empty_like(z)
    iga.iga_kkt_apply(ctx, M, K, beta, z, out)
    b = torch.zeros_like(z)
    bfull = torch.empty(M.info()["n"], dtype=torch.float64, device="cuda")
    load.full(ctx, bfull)
    b[:N] = bfull.reshape(-1)
    rel = float((b - out).norm() / b.norm())
    assert rel <= 1e-6, rel
    print(f"beta {beta}: {info}")
