"""Shared helpers of the GPU parity tests (test side only)."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle.lowrank import band_dense


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def ctx_and_torch():
    torch = require_gpu()
    from paper_1811_06797_gb300 import build, iga
    build.build()
    return iga.Context(), torch, iga


def op_terms(ctx, op):
    """Kronecker terms of a device operator as dense interior matrices (host)."""
    terms = []
    inf = op.info()
    for k in range(inf["nblocks"]):
        R1, R2 = op.block_ranks(k)
        b0, b1, b2 = (op.bands(ctx, k, d) for d in range(3))
        for a in range(R1):
            for c in range(R2):
                terms.append([band_dense(b0[a]), band_dense(b1[a, c]), band_dense(b2[c])])
    return terms


def fro_rel(A, B):
    D = (A - B)
    dn = np.sqrt(D.multiply(D).sum()) if sp.issparse(D) else np.linalg.norm(D)
    bn = np.sqrt(B.multiply(B).sum()) if sp.issparse(B) else np.linalg.norm(B)
    return dn / bn
