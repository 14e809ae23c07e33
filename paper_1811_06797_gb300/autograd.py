"""torch.autograd.Function for the reduced objective of the control problem.

J(u, w) = 1/2 y^T M(w) y - b^T y + beta/2 u^T M(w) u  with  K(w) y = M(w) u,
where w are the univariate weight factors (rank-1 TT cores on the Gauss grid)
of omega and of the six entries of Q.  The forward pass runs the state solve,
the backward pass returns the gradients computed by the library's adjoint
(iga_reduced_gradient: adjoint solve and beta M u - M lam;
iga_weight_gradient: the reverse of the univariate assembly).  All arithmetic
runs in libiga; this module only marshals tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import iga

WEIGHTS = ("omega", "q11", "q12", "q13", "q22", "q23", "q33")


def factor_sizes(space):
    """Gauss-grid lengths (Q1, Q2, Q3) of a space."""
    out = []
    for k in space.knots:
        E = len(np.unique(k)) - 1
        out.append(E * space.nquad)
    return tuple(out)


def geometry_factors(ictx, geometry, space, target, tol):
    """Weight factors (7, Q1+Q2+Q3) of a geometry with rank-1 weights, and the load TT."""
    tts = iga.iga_weight_tts(ictx, geometry, space, target, tol)
    Q = factor_sizes(space)
    w = torch.zeros((7, sum(Q)), dtype=torch.float64, device="cuda")
    for c in range(7):
        t = tts[c]
        if t is None:
            continue
        (_, r) = t.info()
        if r != (1, 1):
            raise iga.IgaError(1, f"weight {WEIGHTS[c]} has TT ranks {r}; rank-1 weights only")
        cores = t.cores(ictx)
        w[c] = torch.tensor(np.concatenate([cores[d].ravel() for d in range(3)]), device="cuda")
    load = iga.iga_load_from_density(ictx, space, tts[7]) if tts[7] is not None else None
    return w, load


def operators_from_factors(ictx, space, w):
    Q = factor_sizes(space)
    off = np.cumsum((0,) + Q)
    tts = []
    for c in range(7):
        if not bool(torch.any(w[c] != 0)):
            tts.append(None)
            continue
        cores = [w[c, off[d]:off[d + 1]].contiguous().view(1, Q[d], 1) for d in range(3)]
        tts.append(iga.iga_tt_from_cores(ictx, cores))
    return iga.iga_ops_from_weights(ictx, space, tts)


class IgaObjective(torch.autograd.Function):
    """J(u, w); gradients with respect to the control u and the weight factors w."""

    @staticmethod
    def forward(fctx, u, w, ictx, space, load, beta, tol):
        M, K = operators_from_factors(ictx, space, w)
        N = u.numel()
        grad_u = torch.empty(N, dtype=torch.float64, device="cuda")
        y = torch.empty(N, dtype=torch.float64, device="cuda")
        lam = torch.empty(N, dtype=torch.float64, device="cuda")
        J = iga.iga_reduced_gradient(ictx, M, K, load, beta, u.detach().contiguous(), grad_u, y, lam,
                                     tol)
        grad_w = torch.empty_like(w)
        iga.iga_weight_gradient(ictx, space, M, K, beta, y, u.detach().contiguous(), lam, grad_w)
        fctx.save_for_backward(grad_u, grad_w)
        return torch.tensor(float(J[0]), dtype=torch.float64, device="cuda")

    @staticmethod
    def backward(fctx, gJ):
        grad_u, grad_w = fctx.saved_tensors
        return gJ * grad_u, gJ * grad_w, None, None, None, None, None


def objective(ictx, space, load, beta, u, w, tol=1e-12):
    return IgaObjective.apply(u, w, ictx, space, load, beta, tol)
