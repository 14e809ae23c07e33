"""Oracle: the KKT solve at grid sizes beyond the sparse direct solve.

Test infrastructure only (see the package header).

The operators come from the oracle's low-rank route (lowrank.weight_tts:
sampled weights on the Gauss grid and TT-SVD, Sec. 3 eq. tt; lowrank_mk and
lowrank_load: univariate factors, Sec. 3 eqs. massFinal / stiffnessFinal),
restricted to the interior (Sec. 4), and applied with
lowrank.kron_apply_modes.  The KKT system (Sec. 4 eq. KKTSystem, one time
step) is solved by kkt.reduced_solve: conjugate gradients on the reduced
system (M + beta K M^{-1} K) y = b, then u = M^{-1} K y, lam = beta u.

M^{-1}: exact per-direction solves when M is one Kronecker term
(M^{-1} = M_1^{-1} (x) M_2^{-1} (x) M_3^{-1}), otherwise an inner conjugate-
gradient solve preconditioned by the inverse of the first term.  The outer
preconditioner is kkt.kron_schur_preconditioner built from the mass factors
of the first M term and the derivative factors of the diagonal stiffness
blocks q_dd, rescaled by the traces of their mass-type factors; it changes
the iteration count, never the solution.

Pins: tests/test_oracle_solve.py checks this route against the sparse direct
solve of the 3-D assembled system on small grids (annulus, twisted annulus,
random volume); the interpolated-weight variant reuses the same solve on the
operators of oracle/interp.py (pinned there).
"""
from __future__ import annotations

import time

import numpy as np

from .assemble import Discretisation
from .kkt import kron_schur_preconditioner, reduced_solve
from .lowrank import kron_apply_modes, lowrank_load, lowrank_operator, restrict_interior, weight_tts


def _inv_term(term):
    inv = [np.linalg.inv(A) for A in term]

    def apply(v):
        return kron_apply_modes([inv], v)
    return apply


def _cg(apply, b, precond, tol):
    x = np.zeros_like(b)
    r = b.copy()
    z = precond(r)
    d = z.copy()
    rz = r @ z
    nb = np.linalg.norm(b)
    it = 0
    while np.linalg.norm(r) > tol * nb and it < 5000:
        Ad = apply(d)
        a = rz / (d @ Ad)
        x += a * d
        r -= a * Ad
        z = precond(r)
        rz2 = r @ z
        d = z + (rz2 / rz) * d
        rz = rz2
        it += 1
    return x


def interior_operators(space, geometry, target, tol, samples=None):
    """Interior Kronecker terms of M and K, the interior load vector and the
    diagonal stiffness terms, from the oracle's low-rank route (`samples`: an
    earlier assemble.sample_weights output of this grid, or None)."""
    disc = Discretisation(space.degree, space.knots, space.nquad)
    return operators_from_tts(space, weight_tts(geometry, disc, tol, target, samples=samples))


def interior_operators_interp(space, geometry, target, tol, pt=None):
    """interior_operators with the weights interpolated in a spline space of
    degree pt (interp.weight_tts_interp) instead of sampled."""
    from .interp import weight_tts_interp
    disc = Discretisation(space.degree, space.knots, space.nquad)
    return operators_from_tts(space, weight_tts_interp(geometry, disc, tol, target, pt))


def operators_from_tts(space, tts):
    """The univariate step alone: interior Kronecker terms of M and K, the
    interior load and the diagonal stiffness terms from weight TT cores
    (lowrank.weight_tts output)."""
    disc = Discretisation(space.degree, space.knots, space.nquad)
    Mt = restrict_interior(lowrank_operator(disc, tts["omega"], "M"))
    kl = {}
    for k in range(3):
        for l in range(3):
            kl[(k, l)] = tts[(min(k, l), max(k, l))]
    Kt = restrict_interior(lowrank_operator(disc, kl, "K"))
    diag = {d: restrict_interior(lowrank_operator(disc, {(d, d): tts[(d, d)]}, "K"))
            for d in range(3) if tts[(d, d)] is not None}
    b = lowrank_load(disc, tts["load"])[1:-1, 1:-1, 1:-1].ravel()
    return Mt, Kt, diag, b


def schur_preconditioner(Mt, diag, beta):
    """kron_schur_preconditioner from the first M term and the first term of
    each diagonal block q_dd (its derivative factor, scaled by the trace
    ratios of its mass-type factors to the M factors)."""
    # the TT-SVD fixes each factor only up to sign: orient every factor to a
    # positive trace (the products are unchanged for a definite operator)
    M1s = [A * np.sign(np.trace(A)) for A in Mt[0]]
    G1s = []
    for d in range(3):
        t = diag[d][0]
        s = 1.0
        for e in range(3):
            if e != d:
                s *= abs(np.trace(t[e])) / np.trace(M1s[e])
        G1s.append(t[d] * np.sign(np.trace(t[d])) * s)
    return kron_schur_preconditioner(M1s, G1s, beta)


def solve_kkt(Mt, Kt, diag, b, beta, tol=1e-12, max_iter=None):
    """(y, u, lam, outer CG iterations) of the stationary KKT system."""
    M_apply = lambda v: kron_apply_modes(Mt, v)
    K_apply = lambda v: kron_apply_modes(Kt, v)
    if len(Mt) == 1:
        Minv = _inv_term(Mt[0])
    else:
        P0 = _inv_term(Mt[0])
        Minv = lambda v: _cg(M_apply, v, P0, 1e-15)
    P = schur_preconditioner(Mt, diag, beta)
    kw = {} if max_iter is None else {"maxit": max_iter}
    return reduced_solve(M_apply, K_apply, Minv, beta, b, tol=tol, precond=P, **kw)


def timed_solve(work, tol=1e-12, tt_tol=None, samples=None):
    """Oracle pipeline on a workload with wall times of its two parts (TT
    truncation at tt_tol, default the workload's)."""
    t0 = time.perf_counter()
    Mt, Kt, diag, b = interior_operators(work.space, work.geometry, work.target,
                                         work.tol if tt_tol is None else tt_tol, samples)
    t1 = time.perf_counter()
    y, u, lam, it = solve_kkt(Mt, Kt, diag, b, work.beta, tol)
    t2 = time.perf_counter()
    return {"y": y, "u": u, "lam": lam, "iters": it, "assembly_s": t1 - t0, "solve_s": t2 - t1,
            "Mt": Mt, "Kt": Kt, "b": b}
