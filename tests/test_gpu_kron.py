"""GPU parity of the Kronecker-sum apply (a5), KKT apply and AMEn local matvec (c)."""
import math

import numpy as np
import pytest

from oracle.amen import local_matvec
from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.kkt import kkt_matrix
from oracle.lowrank import band_dense, kron_apply, kron_matrix
from paper_1811_06797_gb300 import workloads as wl
from gpu_util import ctx_and_torch, op_terms

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _ops(env, name, p, E, tol=1e-12):
    ctx, torch, iga = env
    geo = {"cube": wl.unit_cube(), "annulus": wl.quarter_annulus(),
           "twisted": wl.quarter_annulus(twist=math.pi / 4), "random": wl.random_volume()}[name]
    space = wl.uniform_space(p, E)
    return iga.iga_lowrank_assemble(ctx, geo, space, wl.Target(wl.TARGET_SINPROD), tol)


# n = E + p - 2 unknowns per direction; n = 33 (three 11 x 11 tiles per
# direction) and n = 31 (a 16-wide tile and a ragged 15-wide one) span several
# (i1, i2) tiles
@pytest.mark.parametrize("name,p,E", [("cube", 2, 16), ("annulus", 3, 9), ("twisted", 1, 13),
                                      ("random", 2, 5), ("annulus", 4, 7), ("cube", 2, 33),
                                      ("annulus", 3, 30)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kron_apply(env, name, p, E, prec):
    ctx, torch, iga = env
    M, K, _ = _ops(env, name, p, E, 1e-6 if name == "random" else 1e-12)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(2)
    for op in (M, K):
        terms = op_terms(ctx, op)
        N = int(np.prod(op.info()["n"]))
        x = rng.standard_normal(N)
        y0 = rng.standard_normal(N)
        ref = 0.7 * kron_apply(terms, x) - 1.3 * y0
        xt = torch.tensor(x, device="cuda", dtype=dt)
        yt = torch.tensor(y0, device="cuda", dtype=dt)
        iga.iga_kron_apply(ctx, op, 0.7, xt, -1.3, yt)
        got = yt.double().cpu().numpy()
        tol = 1e-13 if prec == "fp64" else 2e-6
        assert np.linalg.norm(got - ref) < tol * np.linalg.norm(ref)
        # beta = 0 ignores whatever y holds (NaN included)
        yt.fill_(float("nan"))
        iga.iga_kron_apply(ctx, op, 1.0, xt, 0.0, yt)
        assert np.linalg.norm(yt.double().cpu().numpy() - kron_apply(terms, x)) < tol * np.linalg.norm(ref) * 3


@pytest.mark.parametrize("E,tol", [(5, 1e-6), (9, 1e-9)])
def test_ttmatrix_apply_tf32(env, E, tol):
    """Random volume (weight TT ranks > 1): the rank contraction as batched GEMMs,
    FP64 exact, TF32 tensor cores within the TF32 rounding level."""
    ctx, torch, iga = env
    M, K, _ = _ops(env, "random", 2, E, tol)
    assert max(K.info()["R"]) > 3
    rng = np.random.default_rng(9)
    for op in (M, K):
        terms = op_terms(ctx, op)
        N = int(np.prod(op.info()["n"]))
        x = rng.standard_normal(N)
        ref = kron_apply(terms, x)
        y64 = torch.empty(N, dtype=torch.float64, device="cuda")
        iga.iga_kron_apply(ctx, op, 1.0, torch.tensor(x, device="cuda"), 0.0, y64)
        assert np.linalg.norm(y64.cpu().numpy() - ref) < 1e-12 * np.linalg.norm(ref)
        y32 = torch.empty(N, dtype=torch.float32, device="cuda")
        iga.iga_kron_apply(ctx, op, 1.0, torch.tensor(x, device="cuda", dtype=torch.float32), 0.0,
                           y32, tf32=True)
        err = np.linalg.norm(y32.double().cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < 5e-3, err


def test_kkt_apply_against_oracle_assembly(env):
    ctx, torch, iga = env
    work = wl.small(wl.quarter_annulus(twist=math.pi / 4), 2, 5, beta=1e-3)
    M, K, _ = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, 1e-12)
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, _ = assemble_band(work.geometry, disc)
    A = kkt_matrix(band_to_csr(Mb, True), band_to_csr(Kb, True), work.beta)
    z = np.random.default_rng(3).standard_normal(A.shape[0])
    out = torch.empty(A.shape[0], dtype=torch.float64, device="cuda")
    iga.iga_kkt_apply(ctx, M, K, work.beta, torch.tensor(z, device="cuda"), out)
    ref = A @ z
    assert np.linalg.norm(out.cpu().numpy() - ref) < 1e-11 * np.linalg.norm(ref)


@pytest.mark.parametrize("p,E", [(3, 14), (2, 19)])
def test_kkt_apply_fused_rank1(env, p, E):
    """Rank-1 M and K (quarter annulus): the whole KKT operator is one fused
    launch over ragged multi-tile grids, in FP64 and FP32."""
    ctx, torch, iga = env
    work = wl.small(wl.quarter_annulus(), p, E, beta=1e-3)
    M, K, _ = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, 1e-12)
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, _ = assemble_band(work.geometry, disc)
    A = kkt_matrix(band_to_csr(Mb, True), band_to_csr(Kb, True), work.beta)
    z = np.random.default_rng(5).standard_normal(A.shape[0])
    ref = A @ z
    for dt, tol in ((torch.float64, 1e-12), (torch.float32, 5e-6)):
        out = torch.empty(A.shape[0], dtype=dt, device="cuda")
        ctx.profile_begin("kron_rank1_kernel")
        iga.iga_kkt_apply(ctx, M, K, work.beta, torch.tensor(z, device="cuda", dtype=dt), out)
        prof = ctx.profile_end()
        assert prof["launches"] == 1, prof
        err = np.linalg.norm(out.double().cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < tol, (dt, err)


@pytest.mark.parametrize("r0,n,r1,R0,R1,p,nvec", [(1, 17, 5, 1, 3, 2, 3), (6, 11, 7, 3, 2, 3, 2),
                                                 (9, 20, 1, 4, 1, 1, 1), (16, 33, 12, 2, 2, 3, 3)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_local_matvec(env, r0, n, r1, R0, R1, p, nvec, prec):
    ctx, torch, iga = env
    rng = np.random.default_rng(r0 * 100 + r1)
    PhiL = rng.standard_normal((R0, r0, r0))
    PhiR = rng.standard_normal((R1, r1, r1))
    b = 2 * p + 1
    bands = rng.standard_normal((R0, R1, n, b))
    mask = rng.random((R0, R1)) < 0.7
    mask[0, 0] = True
    bands[~mask] = 0.0
    for i in range(n):                 # band entries outside the matrix are zero
        for o in range(b):
            if not 0 <= i + o - p < n:
                bands[:, :, i, o] = 0.0
    x = rng.standard_normal((nvec, r0, n, r1))
    Ad = [[band_dense(bands[a, c]) for c in range(R1)] for a in range(R0)]
    ref = np.stack([local_matvec(PhiL, Ad, PhiR, x[v]) for v in range(nvec)])
    dt = torch.float64 if prec == "fp64" else torch.float32
    T = lambda a: torch.tensor(a, device="cuda", dtype=dt)
    y = torch.empty(x.shape, dtype=dt, device="cuda")
    for m in (None, mask):
        iga.iga_amen_local_matvec(ctx, T(PhiL), T(bands), T(PhiR), T(x), y, bandmask=m)
        tol = 1e-13 if prec == "fp64" else 1e-5
        assert np.linalg.norm(y.double().cpu().numpy() - ref) < tol * np.linalg.norm(ref)


def test_errors_are_reported(env):
    ctx, torch, iga = env
    M, K, _ = _ops(env, "cube", 2, 4)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(iga.IgaError):
        iga.iga_kron_apply(ctx, M, 1.0, x, 0.0, x)      # aliasing rejected
    bad = wl.small(wl.unit_cube(), 2, 4)
    bad.space.knots = (np.array([0, 0, 0.5, 1, 1, 1.0]),) + bad.space.knots[1:]
    with pytest.raises(iga.IgaError) as e:
        iga.iga_lowrank_assemble(ctx, bad.geometry, bad.space, bad.target, 1e-8)
    assert e.value.status == 1 and "end knots" in str(e.value)


def _random_band_op(env, n, p, ranks, seed):
    """Operator from random, non-symmetric banded factors (iga_op_from_bands)
    and its oracle Kronecker terms."""
    ctx, torch, iga = env
    rng = np.random.default_rng(seed)
    b = 2 * p + 1
    blocks, terms = [], []
    for R1, R2 in ranks:
        A1 = rng.standard_normal((R1, n[0], b))
        A2 = rng.standard_normal((R1, R2, n[1], b))
        A3 = rng.standard_normal((R2, n[2], b))
        blocks.append(tuple(torch.tensor(a, device="cuda") for a in (A1, A2, A3)))
        for a in range(R1):
            for c in range(R2):
                terms.append([band_dense(A1[a]), band_dense(A2[a, c]), band_dense(A3[c])])
    return iga.iga_op_from_bands(ctx, blocks), terms


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tf32", "bf16"])
@pytest.mark.parametrize("transpose", [False, True])
def test_operator_from_bands_and_its_transpose(env, prec, transpose):
    """op(A) x for an operator built from random non-symmetric banded factors
    (one rank-1 block and one TT-matrix block), with op(A) = A or A^T (every
    factor transposed, Sec. 5 eq. K_kron), against the oracle's Kronecker
    product of the same (transposed) factors."""
    ctx, torch, iga = env
    n = (23, 19, 21)
    op, terms = _random_band_op(env, n, 2, [(1, 1), (6, 5)], seed=31)
    if transpose:
        terms = [[A.T.copy() for A in t] for t in terms]
    N = int(np.prod(n))
    x = np.random.default_rng(32).standard_normal(N)
    ref = kron_apply(terms, x)
    dt = torch.float64 if prec == "fp64" else torch.float32
    y = torch.zeros(N, dtype=dt, device="cuda")
    iga.iga_kron_apply(ctx, op, 1.0, torch.tensor(x, device="cuda", dtype=dt), 0.0, y,
                       tf32=prec == "tf32", bf16=prec == "bf16", transpose=transpose)
    err = np.linalg.norm(y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < {"fp64": 1e-13, "fp32": 1e-5, "tf32": 5e-3, "bf16": 2.5e-2}[prec], err


@pytest.mark.parametrize("p,E", [(3, 165), (2, 170)])
def test_marching_fp32_apply_on_large_grids(env, p, E):
    """Grids of over 4M points take the marching FP32 kernel (planes
    streamed along i1, modes 3 and 2 in shared memory, mode 1 scattered into
    a register ring): a single operator with beta = 0 and with beta != 0,
    and the whole KKT operator, against the FP64 tiled kernel on the same
    operators, over ragged column tiles and i1 chunks."""
    ctx, torch, iga = env
    work = wl.small(wl.quarter_annulus(twist=np.pi / 4), p, E, beta=1e-3)
    M, K, _ = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, 1e-10)
    N = int(np.prod(M.info()["n"]))
    assert N >= 4194304
    g = torch.Generator(device="cuda").manual_seed(E)
    x = torch.randn(N, generator=g, device="cuda", dtype=torch.float64)
    y0 = torch.randn(N, generator=g, device="cuda", dtype=torch.float64)
    for op in (M, K):
        for beta in (0.0, -0.5):
            ref = y0.clone()
            iga.iga_kron_apply(ctx, op, 1.5, x, beta, ref)
            y32 = y0.float()
            ctx.profile_begin("kron_march_kernel")
            iga.iga_kron_apply(ctx, op, 1.5, x.float(), beta, y32)
            prof = ctx.profile_end()
            assert prof["launches"] >= 1, prof
            err = float((y32.double() - ref).norm() / ref.norm())
            assert err < 1e-5, (beta, err)
    z = torch.randn(3 * N, generator=g, device="cuda", dtype=torch.float64)
    ref = torch.empty_like(z)
    iga.iga_kkt_apply(ctx, M, K, work.beta, z, ref)
    out = torch.empty(3 * N, device="cuda", dtype=torch.float32)
    ctx.profile_begin("kron_march_kernel")
    iga.iga_kkt_apply(ctx, M, K, work.beta, z.float(), out)
    prof = ctx.profile_end()
    assert prof["launches"] == 1, prof
    err = float((out.double() - ref).norm() / ref.norm())
    assert err < 1e-5, err
