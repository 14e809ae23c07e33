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
