"""The allocation-free local matvec (iga_amen_local_matvec_noalloc).

It serves callers that cannot allocate device memory: it must give the same
result as iga_amen_local_matvec while using only the library's fixed device
scratch.  This file is collected last so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

from gpu_util import ctx_and_torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _case(rng, r0, n, r1, R0, R1, p, nvec, dt, torch, masked):
    b = 2 * p + 1
    PhiL = rng.standard_normal((R0, r0, r0))
    PhiR = rng.standard_normal((R1, r1, r1))
    bands = rng.standard_normal((R0, R1, n, b))
    mask = None
    if masked:
        mask = rng.random((R0, R1)) < 0.6
        mask[0, 0] = True
        bands[~mask] = 0.0
    for i in range(n):
        for o in range(b):
            if not 0 <= i + o - p < n:
                bands[:, :, i, o] = 0.0
    x = rng.standard_normal((nvec, r0, n, r1))
    T = lambda a: torch.tensor(a, device="cuda", dtype=dt)
    return T(PhiL), T(bands), T(PhiR), T(x), mask


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_matches_allocating_entry_point_twice(env, prec):
    ctx, torch, iga = env
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-13 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(11)
    shapes = [(7, 23, 9, 3, 2, 3, 3, True), (12, 40, 5, 1, 4, 2, 2, False)]
    cases = [_case(rng, *s[:7], dt, torch, s[7]) for s in shapes]
    outs = [torch.empty(c[3].shape, dtype=dt, device="cuda") for c in cases]
    refs = [torch.empty(c[3].shape, dtype=dt, device="cuda") for c in cases]
    for (PhiL, bands, PhiR, x, mask), ref in zip(cases, refs):
        iga.iga_amen_local_matvec(ctx, PhiL, bands, PhiR, x, ref, bandmask=mask)
    torch.cuda.synchronize()
    # first call on the device does the one-time address lookup
    iga.iga_amen_local_matvec_noalloc(*cases[0][:4], outs[0], bandmask=cases[0][4])
    for out in outs:
        out.fill_(float("nan"))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    # two calls in a row, each checked against the allocating entry point
    for (PhiL, bands, PhiR, x, mask), out, ref in zip(cases, outs, refs):
        iga.iga_amen_local_matvec_noalloc(PhiL, bands, PhiR, x, out, bandmask=mask)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0          # nothing was allocated
    for out, ref in zip(outs, refs):
        err = (out.double() - ref.double()).norm() / ref.double().norm()
        assert float(err) < tol, float(err)


def test_noalloc_rejects_sizes_beyond_its_scratch(env):
    ctx, torch, iga = env
    # (R0 + R1) * nvec * r0 * n * r1 * 8 bytes = 2 * 3 * 64 * 100 * 64 * 8 > 16 MiB
    PhiL = torch.zeros((1, 64, 64), dtype=torch.float64, device="cuda")
    PhiR = torch.zeros((1, 64, 64), dtype=torch.float64, device="cuda")
    bands = torch.zeros((1, 1, 100, 7), dtype=torch.float64, device="cuda")
    x = torch.zeros((3, 64, 100, 64), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(iga.IgaError) as e:
        iga.iga_amen_local_matvec_noalloc(PhiL, bands, PhiR, x, y)
    assert e.value.status == 1


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_noalloc_on_a_side_stream_with_two_different_masks(env, prec):
    # the shared mask buffer is safe only through stream order: two masked
    # calls in a row on one non-default stream, each with its own mask
    ctx, torch, iga = env
    dt = torch.float64 if prec == "fp64" else torch.float32
    tol = 1e-13 if prec == "fp64" else 1e-5
    rng = np.random.default_rng(12)
    cases = [_case(rng, 5, 19, 6, 3, 4, 2, 2, dt, torch, True),
             _case(rng, 5, 19, 6, 3, 4, 2, 2, dt, torch, True)]
    assert not np.array_equal(cases[0][4], cases[1][4])
    refs = [torch.empty(c[3].shape, dtype=dt, device="cuda") for c in cases]
    for (PhiL, bands, PhiR, x, mask), ref in zip(cases, refs):
        iga.iga_amen_local_matvec(ctx, PhiL, bands, PhiR, x, ref, bandmask=mask)
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    outs = [torch.full(c[3].shape, float("nan"), dtype=dt, device="cuda") for c in cases]
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for (PhiL, bands, PhiR, x, mask), out in zip(cases, outs):
            iga.iga_amen_local_matvec_noalloc(PhiL, bands, PhiR, x, out, bandmask=mask,
                                              stream=side)
    side.synchronize()
    for out, ref in zip(outs, refs):
        err = (out.double() - ref.double()).norm() / ref.double().norm()
        assert float(err) < tol, float(err)
