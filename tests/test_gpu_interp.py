"""The paper's weight-interpolation route on the GPU (iga_weight_tts_interp,
iga_lowrank_assemble_interp; Sec. 3 eqs. weightEquationSystem and
weightEquationSolve) against the oracle's own interpolation route
(oracle/interp.py): the weight TTs at the Gauss points and the assembled
operators, element by element."""
import math

import numpy as np
import pytest

from gpu_util import ctx_and_torch, op_terms
from oracle.assemble import Discretisation
from oracle.interp import weight_tts_interp
from oracle.lowrank import kron_matrix, lowrank_mk, restrict_interior, tt_full
from paper_1811_06797_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

NAMES = ["omega", (0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2), "load"]


@pytest.fixture(scope="module")
def env():
    return ctx_and_torch()


def _dense(ctx, tt, torch):
    if tt is None:
        return None
    n, _ = tt.info()
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    tt.full(ctx, out)
    return out.cpu().numpy()


CASES = {"annulus": (wl.quarter_annulus(), 2, 6), "twisted": (wl.quarter_annulus(twist=math.pi / 4), 3, 4),
         "random": (wl.random_volume(), 2, 5)}


@pytest.mark.parametrize("name", list(CASES))
def test_interpolated_weights_match_the_oracle(env, name):
    ctx, torch, iga = env
    geo, p, E = CASES[name]
    target = wl.Target(wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1)
    space = wl.uniform_space(p, E)
    disc = Discretisation(space.degree, space.knots, space.nquad)
    got = iga.iga_weight_tts_interp(ctx, geo, space, target, 1e-13)
    ref = weight_tts_interp(geo, disc, 1e-13, target)
    qref = math.sqrt(sum((2 if k != l else 1) * np.linalg.norm(tt_full(ref[(k, l)])) ** 2
                         for k in range(3) for l in range(k, 3) if ref[(k, l)] is not None))
    for c, key in enumerate(NAMES):
        g = _dense(ctx, got[c], torch)
        r = tt_full(ref[key]) if ref[key] is not None else None
        scale = qref if isinstance(key, tuple) else np.linalg.norm(r)
        if r is None or np.linalg.norm(r) < 1e-12 * scale:
            assert g is None or np.linalg.norm(g) < 1e-11 * scale, key
            continue
        assert g is not None, key
        assert np.linalg.norm(g - r) < 1e-10 * scale, (key, np.linalg.norm(g - r) / scale)


def test_interpolated_operators_match_the_oracle(env):
    ctx, torch, iga = env
    geo, p, E = CASES["random"]
    space = wl.uniform_space(p, E)
    disc = Discretisation(space.degree, space.knots, space.nquad)
    M, K, _ = iga.iga_lowrank_assemble_interp(ctx, geo, space, None, 1e-12)
    Mt, Kt = lowrank_mk(disc, weight_tts_interp(geo, disc, 1e-12))
    for op, terms in ((M, Mt), (K, Kt)):
        A = kron_matrix(op_terms(ctx, op))
        B = kron_matrix(restrict_interior(terms))
        diff = A - B
        assert np.sqrt(diff.multiply(diff).sum()) < 1e-9 * np.sqrt(B.multiply(B).sum())
