"""Rank and storage reporting (the quantities of the paper's rank tables,
Sec. 6, Tables ranks1 / ranks2 / ranks3, and its storage comparison of the
low-rank factors with the assembled sparse matrices).

Everything here is read from the library through the C ABI: the TT ranks of
the sampled weights (iga_weight_tts) and the device bytes of the assembled
Kronecker / TT-matrix factors (iga_op_info).  The CSR size of the assembled
3-D matrix is a count: row i of a degree-p B-spline matrix has one nonzero
for every basis function whose support overlaps that of basis function i,
i.e. prod_d (number of j_d with |i_d - j_d| <= p inside the index range).
"""
from __future__ import annotations

from . import iga

WEIGHT_NAMES = ("omega", "q11", "q12", "q13", "q22", "q23", "q33")


def csr_nnz(n, p):
    """Nonzeros of the Dirichlet-reduced 3-D matrix with n[d] interior
    functions of degree p[d] per direction (full band pattern)."""
    nnz = 1
    for nd, pd in zip(n, p):
        # sum over rows of the number of columns within distance pd
        s = 0
        for i in range(nd):
            s += min(nd - 1, i + pd) - max(0, i - pd) + 1
        nnz *= s
    return nnz


def rank_table(ctx, geometry, space, tols):
    """{tol: {weight: (R1, R2) or None}} for the seven sampled weights."""
    out = {}
    for tol in tols:
        tts = iga.iga_weight_tts(ctx, geometry, space, None, tol)
        out[tol] = {name: (tts[c].info()[1] if tts[c] is not None else None)
                    for c, name in enumerate(WEIGHT_NAMES)}
    return out


def storage(ctx, geometry, space, target, tol):
    """Bytes of the low-rank M and K factors (FP64 and the FP32 copy) against
    the CSR storage of the assembled matrices (8-byte values, 4-byte column
    indices, 8-byte row offsets)."""
    M, K, _ = iga.iga_lowrank_assemble(ctx, geometry, space, target, tol)
    res = {}
    for name, op in (("M", M), ("K", K)):
        inf = op.info()
        nnz = csr_nnz(inf["n"], inf["p"])
        N = inf["n"][0] * inf["n"][1] * inf["n"][2]
        res[name] = {"factor_bytes": inf["bytes"], "blocks": inf["nblocks"], "R": inf["R"],
                     "csr_nnz": nnz, "csr_bytes": 12 * nnz + 8 * (N + 1)}
    return res
