"""Boundary behaviour of the C ABI: TT files, the TT-valued solve, and the
errors a caller can provoke from the host (an allocation that cannot be
served, a degenerate or folded geometry).  No test faults the GPU: the
allocation failure is a request larger than the device, refused before any
kernel runs, and the geometry errors are flags the sampling kernel sets."""
import math

import numpy as np
import pytest

from gpu_util import ctx_and_torch
from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.geometry import map_and_jacobian
from oracle.kkt import kkt_solve
from paper_1811_06797_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def test_tt_save_load_roundtrip(env, tmp_path):
    ctx, torch, iga = env
    rng = np.random.default_rng(3)
    cores = [rng.standard_normal(s) for s in ((1, 7, 3), (3, 5, 4), (4, 6, 1))]
    tt = iga.iga_tt_from_cores(ctx, [torch.tensor(c, device="cuda") for c in cores])
    path = tmp_path / "w.igatt"
    tt.save(ctx, path)
    assert path.stat().st_size == 8 + 5 * 4 + 8 * sum(c.size for c in cores)
    back = iga.iga_tt_load(ctx, path)
    assert back.info() == ((7, 5, 6), (3, 4))
    for d in range(3):
        assert np.array_equal(back.core(ctx, d), cores[d])
    full = torch.empty((7, 5, 6), dtype=torch.float64, device="cuda")
    back.full(ctx, full)
    ref = np.einsum("xia,ajb,bky->ijk", *cores)
    assert np.allclose(full.cpu().numpy(), ref, rtol=0, atol=1e-12)
    # a truncated file, a wrong magic and a missing file are refused
    raw = path.read_bytes()
    bad = tmp_path / "bad.igatt"
    bad.write_bytes(raw[:-8])
    with pytest.raises(iga.IgaError) as e:
        iga.iga_tt_load(ctx, bad)
    assert e.value.status == 1
    bad.write_bytes(b"NOTATT!!" + raw[8:])
    with pytest.raises(iga.IgaError):
        iga.iga_tt_load(ctx, bad)
    with pytest.raises(iga.IgaError):
        iga.iga_tt_load(ctx, tmp_path / "missing.igatt")


def test_solve_with_tt_outputs_matches_the_direct_solve(env):
    ctx, torch, iga = env
    work = wl.small(wl.quarter_annulus(), 2, 6,
                    wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1), beta=1e-3, tol=1e-12)
    M, K, load = iga.iga_lowrank_assemble(ctx, work.geometry, work.space, work.target, work.tol)
    y, u, lam, info = iga.iga_kkt_solve_amen_tt(ctx, M, K, load, work.beta, tol=1e-9)
    assert info["converged"], info
    disc = Discretisation(work.space.degree, work.space.knots, work.space.nquad)
    Mb, Kb, b = assemble_band(work.geometry, disc, work.target)
    ref = kkt_solve(band_to_csr(Mb, True), band_to_csr(Kb, True), work.beta,
                    b[1:-1, 1:-1, 1:-1].ravel())
    n = M.info()["n"]
    for tt, r in zip((y, u, lam), ref):
        assert tt.info()[0] == n
        full = torch.empty(n, dtype=torch.float64, device="cuda")
        tt.full(ctx, full)
        err = np.linalg.norm(full.cpu().numpy().ravel() - r) / np.linalg.norm(r)
        assert err < 1e-7, err


def test_allocation_beyond_the_device_gives_enomem_and_the_context_survives(env):
    ctx, torch, iga = env
    # a TT-matrix block whose FP64 apply stages (n2 + 2p) R2 n1 n3 doubles:
    # 10 x 6000 x 2^20 x 8 B = 503 GB, more than any GB300 holds; the request
    # is refused before any kernel runs
    n1, n2, n3, R2 = 1024, 8, 1024, 6000
    A1 = torch.zeros((1, n1, 3), dtype=torch.float64, device="cuda")
    A1[:, :, 1] = 1.0
    A2 = torch.zeros((1, R2, n2, 3), dtype=torch.float64, device="cuda")
    A2[:, :, :, 1] = 1.0
    A3 = torch.zeros((R2, n3, 3), dtype=torch.float64, device="cuda")
    A3[:, :, 1] = 1.0
    op = iga.iga_op_from_bands(ctx, [(A1, A2, A3)])
    x = torch.ones(n1 * n2 * n3, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(iga.IgaError) as e:
        iga.iga_kron_apply(ctx, op, 1.0, x, 0.0, y)
    assert e.value.status == 2, e.value                       # IGA_ENOMEM
    del op, A2, A3
    # the context still works
    small = iga.iga_op_from_bands(ctx, [(A1[:, :16].contiguous(),
                                          torch.ones((1, 1, 4, 3), dtype=torch.float64,
                                                     device="cuda"),
                                          torch.ones((1, 5, 3), dtype=torch.float64,
                                                     device="cuda"))])
    xs = torch.ones(16 * 4 * 5, dtype=torch.float64, device="cuda")
    ys = torch.empty_like(xs)
    iga.iga_kron_apply(ctx, small, 1.0, xs, 0.0, ys)
    torch.cuda.synchronize()
    # A1 = I and the other two factors are tridiagonal all-ones: interior
    # entries of the product are 3 x 3 = 9
    assert float(ys.reshape(16, 4, 5)[3, 1, 2]) == 9.0


def _cubic_box(xs):
    """Degree-3 B-spline map with 4 control points per direction, identity in
    y and z and control x-coordinates xs in direction 1."""
    k = wl.open_uniform_knots(3, 1)
    g = wl.greville(k, 3)
    c = np.stack(np.meshgrid(np.asarray(xs, float), g, g, indexing="ij"), axis=-1)
    return wl.Geometry(wl.GEO_NURBS, (3, 3, 3), (k, k.copy(), k.copy()), c, np.ones(c.shape[:3]))


def test_degenerate_and_folded_geometries_are_rejected(env):
    ctx, torch, iga = env
    space = wl.uniform_space(2, 4)
    Q = 4 * space.nquad
    out = torch.empty(8 * Q ** 3, dtype=torch.float64, device="cuda")
    # folded: control x-coordinates 0, 1.2, -0.2, 1 make dx/dxhat change sign
    # (x'(1/2) = 3 (0.3 - 0.7 + 0.3) < 0 < x'(0))
    folded = _cubic_box([0.0, 1.2, -0.2, 1.0])
    disc = Discretisation(space.degree, space.knots, space.nquad)
    pts = np.array([[t, 0.5, 0.5] for t in disc.x[0].ravel()])
    _, J = map_and_jacobian(folded.kind, folded.degree, folded.knots, folded.homogeneous(), 0.0, pts)
    dets = np.linalg.det(J)
    assert dets.min() < 0 < dets.max()                       # the oracle sees the fold
    with pytest.raises(iga.IgaError) as e:
        iga.iga_sample_weights(ctx, folded, space, None, out)
    assert e.value.status == 1 and "sign" in str(e.value)
    # degenerate: every control point equal in x
    flat = _cubic_box([0.5, 0.5, 0.5, 0.5])
    with pytest.raises(iga.IgaError) as e:
        iga.iga_sample_weights(ctx, flat, space, None, out)
    assert e.value.status == 1
    # a mirrored (left-handed) map is a valid domain: omega = |det J| is the
    # same as for the right-handed one
    right = _cubic_box([0.0, 1 / 3, 2 / 3, 1.0])
    left = _cubic_box([1.0, 2 / 3, 1 / 3, 0.0])
    a = torch.empty_like(out)
    iga.iga_sample_weights(ctx, right, space, None, a)
    iga.iga_sample_weights(ctx, left, space, None, out)
    om_r = a[:Q ** 3].reshape(Q, Q, Q)
    om_l = out[:Q ** 3].reshape(Q, Q, Q)
    assert torch.allclose(om_l, om_r.flip(0), rtol=1e-13, atol=0)
