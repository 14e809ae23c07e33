"""TT-matrix Kronecker apply with the rank contraction on the tensor cores.

Blocks with TT ranks above one (Sec. 5, eq. K_kron) in FP32 storage run the
fused tcgen05 kernel: mode-3 slabs in shared memory, the dense rank
contraction as TF32 MMAs accumulated in tensor memory, the mode-1 product in
the epilogue.  Random weight TTs of chosen ranks give operators whose shapes
cover one and two tensor-memory halves, ragged tiles in i1 and i3, grids
smaller than the band and ranks that are not multiples of the MMA sizes.
The reference is the oracle's Kronecker product of the operator's own factors
(FP64, by definition); the bound is the TF32 rounding level."""
import numpy as np
import pytest

from gpu_util import ctx_and_torch, op_terms
from oracle.lowrank import kron_apply_modes
from paper_1811_06797_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def random_op(env, p, E, R1, R2, seed):
    ctx, torch, iga = env
    space = wl.uniform_space(p, E)
    Q = E * space.nquad
    rng = np.random.default_rng(seed)
    cores = [rng.uniform(0.5, 1.5, (1, Q, R1)), rng.standard_normal((R1, Q, R2)),
             rng.uniform(0.5, 1.5, (R2, Q, 1))]
    tt = iga.iga_tt_from_cores(ctx, [torch.tensor(c, device="cuda") for c in cores])
    M, _ = iga.iga_ops_from_weights(ctx, space, [tt] + [None] * 6)
    return M


CASES = [(2, 13, 7, 5), (1, 22, 17, 9), (3, 9, 12, 20), (2, 30, 35, 33), (2, 21, 48, 48),
         (2, 2, 4, 3), (3, 5, 40, 8), (2, 41, 16, 24)]
# operand rounding: TF32 keeps 10 fraction bits, BF16 7 (relative 2^-11 and
# 2^-8 per operand, round to nearest); the bounds leave room for a sum of a
# few hundred such products
TOL = {"tf32": (5e-3, 2e-2), "bf16": (2.5e-2, 8e-2)}


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
@pytest.mark.parametrize("p,E,R1,R2", CASES)
def test_tensor_core_apply_matches_the_kronecker_definition(env, p, E, R1, R2, kind):
    ctx, torch, iga = env
    M = random_op(env, p, E, R1, R2, seed=R1 * 100 + R2)
    assert M.block_ranks(0) == (R1, R2)
    n = M.info()["n"]
    N = int(np.prod(n))
    rng = np.random.default_rng(E)
    x = rng.standard_normal(N)
    y0 = rng.standard_normal(N)
    ref = kron_apply_modes(op_terms(ctx, M), x)
    xt = torch.tensor(x, device="cuda", dtype=torch.float32)
    yt = torch.tensor(y0, device="cuda", dtype=torch.float32)
    ctx.profile_begin("ttm_tc_kernel")
    iga.iga_kron_apply(ctx, M, 0.75, xt, 0.5, yt, tf32=kind == "tf32", bf16=kind == "bf16")
    prof = ctx.profile_end()
    assert prof["launches"] == 1                      # the fused tensor-core kernel ran
    want = 0.75 * ref + 0.5 * y0
    got = yt.double().cpu().numpy()
    err = np.linalg.norm(got - want) / np.linalg.norm(want)
    tn, tm = TOL[kind]
    assert err < tn, err
    assert np.abs(got - want).max() < tm * np.abs(want).max()


@pytest.mark.parametrize("kind", ["tf32", "bf16"])
def test_tensor_core_apply_is_deterministic_and_accumulates(env, kind):
    ctx, torch, iga = env
    M = random_op(env, 2, 17, 20, 20, seed=5)
    N = int(np.prod(M.info()["n"]))
    x = torch.randn(N, device="cuda", dtype=torch.float32)
    y1 = torch.zeros(N, device="cuda", dtype=torch.float32)
    y2 = torch.zeros(N, device="cuda", dtype=torch.float32)
    kw = {kind: True}
    iga.iga_kron_apply(ctx, M, 1.0, x, 0.0, y1, **kw)
    iga.iga_kron_apply(ctx, M, 1.0, x, 0.0, y2, **kw)
    assert torch.equal(y1, y2)
    # y = 2 A x from two accumulating calls equals one call with alpha = 2
    iga.iga_kron_apply(ctx, M, 1.0, x, 1.0, y2, **kw)
    y3 = torch.zeros(N, device="cuda", dtype=torch.float32)
    iga.iga_kron_apply(ctx, M, 2.0, x, 0.0, y3, **kw)
    assert float((y2 - y3).abs().max()) <= 1e-5 * float(y3.abs().max())
