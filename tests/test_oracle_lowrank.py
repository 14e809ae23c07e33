"""Pins of the oracle's TT-SVD, univariate factors and Kronecker apply."""
import json
import math
import os

import numpy as np
import pytest

from oracle.assemble import Discretisation, assemble_band, band_to_csr
from oracle.lowrank import (kron_apply, kron_matrix, lowrank_load, lowrank_mk, restrict_interior,
                            tt_full, tt_ranks, tt_svd, weight_tts)
from paper_1811_06797_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _random_tt(n, r, seed):
    rng = np.random.default_rng(seed)
    ranks = (1,) + tuple(r) + (1,)
    return [rng.standard_normal((ranks[d], n[d], ranks[d + 1])) for d in range(3)]


def test_tt_svd_exact_rank():
    cores = _random_tt((7, 9, 8), (3, 4), 0)
    W = tt_full(cores)
    out = tt_svd(W, 1e-12)
    assert tt_ranks(out) == (3, 4)
    assert np.linalg.norm(tt_full(out) - W) < 1e-12 * np.linalg.norm(W)


@pytest.mark.parametrize("tol", [1e-1, 1e-2, 1e-4])
def test_tt_svd_error_bound(tol):
    W = np.random.default_rng(1).standard_normal((10, 11, 12))
    out = tt_svd(W, tol)
    err = np.linalg.norm(tt_full(out) - W) / np.linalg.norm(W)
    assert err <= tol * (1 + 1e-12)
    # the rank is not larger than needed: one rank less in the first unfolding breaks the bound
    r1, r2 = tt_ranks(out)
    if r1 > 1:
        worse = tt_svd(W, tol, rmax=r1 - 1)
        assert np.linalg.norm(tt_full(worse) - W) / np.linalg.norm(W) > tol / math.sqrt(2) * 0.999


def test_tt_svd_threshold_splits_the_budget():
    """The tolerance is split over the D - 1 = 2 unfoldings (threshold
    tol ||W|| / sqrt(2) each, Sec. 3).  W = a b c + e a' b' c + e a b'' c'
    with orthonormal a, a' and b, b', b'' and c, c' has one singular value e
    in the tail of each unfolding.  With e = 0.9 tol both must be kept
    (0.9 > 1/sqrt(2)); a threshold of tol per unfolding would drop both and
    leave an error of 1.27 tol."""
    rng = np.random.default_rng(5)
    qa, _ = np.linalg.qr(rng.standard_normal((6, 2)))
    qb, _ = np.linalg.qr(rng.standard_normal((4, 3)))
    qc, _ = np.linalg.qr(rng.standard_normal((5, 2)))
    tol = 1e-3
    e = 0.9 * tol
    outer = lambda x, y, z: np.einsum("i,j,k->ijk", x, y, z)
    W = (outer(qa[:, 0], qb[:, 0], qc[:, 0]) + e * outer(qa[:, 1], qb[:, 1], qc[:, 0])
         + e * outer(qa[:, 0], qb[:, 2], qc[:, 1]))
    out = tt_svd(W, tol)
    err = np.linalg.norm(tt_full(out) - W) / np.linalg.norm(W)
    assert err <= tol
    assert tt_ranks(out) == (2, 2)


def test_tt_svd_separable_and_zero():
    a, b, c = (np.random.default_rng(2).standard_normal(m) for m in (5, 6, 7))
    W = np.einsum("i,j,k->ijk", a, b, c)
    assert tt_ranks(tt_svd(W, 1e-14)) == (1, 1)
    assert tt_svd(np.zeros((3, 3, 3)), 1e-8) is None
    assert tt_svd(1e-20 * W, 1e-8, norm=1.0) is None


def test_kron_apply_definition_tiny():
    rng = np.random.default_rng(3)
    terms = [[rng.standard_normal((m, m)) for m in (3, 4, 2)] for _ in range(2)]
    x = rng.standard_normal(24)
    dense = sum(np.kron(t[0], np.kron(t[1], t[2])) for t in terms)
    assert np.allclose(kron_apply(terms, x), dense @ x, atol=1e-13)


def _fro_rel(A, B):
    return np.linalg.norm((A - B).data if hasattr(A - B, "data") else A - B) / np.linalg.norm(
        B.data if hasattr(B, "data") else B)


@pytest.mark.parametrize("name,geo", [("cube", wl.unit_cube()), ("annulus", wl.quarter_annulus())])
def test_univariate_route_exact_on_rank_one_geometry(name, geo):
    space = wl.uniform_space(2, 4)
    disc = Discretisation(space.degree, space.knots, space.nquad)
    tgt = wl.Target(wl.TARGET_SINPROD) if name == "cube" else wl.Target(
        wl.TARGET_GAUSS, wl.ANNULUS_CENTROID, 0.1)
    Mb, Kb, b = assemble_band(geo, disc, tgt)
    tts = weight_tts(geo, disc, 1e-13, tgt)
    Mt, Kt = lowrank_mk(disc, tts)
    assert _fro_rel(kron_matrix(Mt), band_to_csr(Mb)) < 1e-13
    assert _fro_rel(kron_matrix(Kt), band_to_csr(Kb)) < 1e-12
    bl = lowrank_load(disc, tts["load"])
    assert np.linalg.norm(bl - b) < 1e-12 * np.linalg.norm(b)
    if name == "cube":
        assert tt_ranks(tts["load"]) == (1, 1)


def test_annulus_ranks_golden():
    gold = json.load(open(os.path.join(GOLD, "annulus_weight_ranks.json")))
    space = wl.uniform_space(3, 8)
    disc = Discretisation(space.degree, space.knots, space.nquad)
    tts = weight_tts(wl.quarter_annulus(), disc, 1e-10)
    names = {"omega": "omega", "q11": (0, 0), "q22": (1, 1), "q33": (2, 2),
             "q12": (0, 1), "q13": (0, 2), "q23": (1, 2)}
    for key, r in gold["ranks"].items():
        assert list(tt_ranks(tts[names[key]])) == r, key
    for key in gold["rank0"]:
        assert tts[names[key]] is None, key


def test_twisted_annulus_within_truncation_tolerance():
    geo = wl.quarter_annulus(twist=math.pi / 4)
    space = wl.uniform_space(2, 5)
    disc = Discretisation(space.degree, space.knots, space.nquad)
    _, Kb, _ = assemble_band(geo, disc)
    K = band_to_csr(Kb, interior=True)
    for tol in (1e-4, 1e-7):
        tts = weight_tts(geo, disc, tol)
        _, Kt = lowrank_mk(disc, tts)
        err = _fro_rel(kron_matrix(restrict_interior(Kt)), K)
        assert err < 10 * tol, (tol, err)
    # the twist couples the angular and axial directions (q13 != 0), but the
    # metric does not depend on z, so every weight keeps TT rank 1
    assert tts[(0, 2)] is not None and tt_ranks(tts[(0, 2)]) == (1, 1)
    assert tts[(0, 1)] is None and tts[(1, 2)] is None


def test_random_volume_high_rank_within_tolerance():
    geo = wl.random_volume()
    space = wl.uniform_space(2, 5)
    disc = Discretisation(space.degree, space.knots, space.nquad)
    Mb, Kb, _ = assemble_band(geo, disc)
    for tol in (1e-3, 1e-6):
        tts = weight_tts(geo, disc, tol)
        Mt, Kt = lowrank_mk(disc, tts)
        assert _fro_rel(kron_matrix(Mt), band_to_csr(Mb)) < 10 * tol
        assert _fro_rel(kron_matrix(Kt), band_to_csr(Kb)) < 10 * tol
    assert min(tt_ranks(tts["omega"])) > 3


def test_kron_apply_modes_equals_the_sparse_definition():
    from oracle.lowrank import kron_apply_modes
    rng = np.random.default_rng(4)
    terms = [[rng.standard_normal((m, m)) for m in (5, 3, 4)] for _ in range(3)]
    x = rng.standard_normal(60)
    assert np.allclose(kron_apply_modes(terms, x), kron_apply(terms, x), rtol=0, atol=1e-12)
    dense = sum(np.kron(t[0], np.kron(t[1], t[2])) for t in terms)
    assert np.allclose(kron_apply_modes(terms, x), dense @ x, atol=1e-12)
