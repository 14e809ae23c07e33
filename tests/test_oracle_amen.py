"""Pins of the oracle's frame matrix and projected (local) operators."""
import numpy as np
import pytest

from oracle.amen import (frame_matrix, interfaces, local_kkt_frame, local_matvec,
                         local_operator_frame, local_operator_interfaces)


def _cores(n, r, seed, orth_center=None):
    rng = np.random.default_rng(seed)
    ranks = (1,) + tuple(r) + (1,)
    cores = [rng.standard_normal((ranks[d], n[d], ranks[d + 1])) for d in range(3)]
    if orth_center is not None:
        d0 = orth_center
        for d in range(d0):                      # left-orthonormal cores
            C = cores[d].reshape(-1, ranks[d + 1])
            Q, _ = np.linalg.qr(C)
            cores[d] = Q.reshape(cores[d].shape)
        for d in range(2, d0, -1):               # right-orthonormal cores
            C = cores[d].reshape(ranks[d], -1).T
            Q, _ = np.linalg.qr(C)
            cores[d] = Q.T.reshape(cores[d].shape)
    return cores


def _op(n, R, seed):
    rng = np.random.default_rng(seed)
    A1 = [rng.standard_normal((n[0], n[0])) for _ in range(R[0])]
    A2 = [[rng.standard_normal((n[1], n[1])) for _ in range(R[1])] for _ in range(R[0])]
    A3 = [rng.standard_normal((n[2], n[2])) for _ in range(R[1])]
    return A1, A2, A3


@pytest.mark.parametrize("d", [0, 1, 2])
def test_interfaces_equal_frame_projection(d):
    n, r, R = (4, 5, 3), (2, 3), (2, 3)
    cores = _cores(n, r, d)
    op = _op(n, R, 10 + d)
    PhiL, Ad, PhiR = interfaces(op, cores, d)
    A_if = local_operator_interfaces(PhiL, Ad, PhiR)
    A_fr = local_operator_frame(op, cores, d)
    assert np.allclose(A_if, A_fr, atol=1e-11 * np.abs(A_fr).max())
    x = np.random.default_rng(5).standard_normal(A_fr.shape[0])
    rl = (1, r[0], r[1], 1)
    xs = x.reshape(rl[d], n[d], rl[d + 1])
    assert np.allclose(local_matvec(PhiL, Ad, PhiR, xs).ravel(), A_fr @ x,
                       atol=1e-11 * np.abs(A_fr).max())


@pytest.mark.parametrize("d", [0, 1, 2])
def test_orthonormal_frame(d):
    cores = _cores((4, 5, 3), (2, 3), 7, orth_center=d)
    F = frame_matrix(cores, d)
    assert np.allclose(F.T @ F, np.eye(F.shape[1]), atol=1e-13)


def test_local_kkt_blocks():
    n, r = (3, 4, 3), (2, 2)
    cores = _cores(n, r, 1, orth_center=1)
    opM = _op(n, (1, 1), 2)
    opK = _op(n, (2, 1), 3)
    beta = 0.5
    A = local_kkt_frame(opM, opK, beta, cores, 1)
    m = r[0] * n[1] * r[1]
    Mloc = local_operator_frame(opM, cores, 1)
    assert np.allclose(A[:m, :m], Mloc) and np.allclose(A[m:2 * m, m:2 * m], beta * Mloc)
    assert np.allclose(A[2 * m:, :m], local_operator_frame(opK, cores, 1))
    assert np.allclose(A[:m, 2 * m:], A[2 * m:, :m].T)
