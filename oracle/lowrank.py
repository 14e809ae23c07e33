"""Oracle: TT-SVD, univariate factor assembly, Kronecker-sum apply.

Test infrastructure only (see the package header).

  tt_svd           -- Sec. 3 eq. tt: W(i1,i2,i3) = W_1(i1) W_2(i2) W_3(i3),
                      computed by sequential truncated SVDs of the
                      unfoldings (TT-SVD, cited in Sec. 3 after eq.
                      weightEquationSolve), threshold tol ||W||_F / sqrt(D-1)
                      per unfolding.
  univariate_band  -- Sec. 3 eqs. massMatrix1D and the univariate stiffness
                      matrices K_kl^(d): int (delta(l,d) B) (x) (delta(k,d) B) q dx,
                      with the weight known at the Gauss points of the
                      discretisation (it is sampled there, with the Gauss
                      weights folded in).
  lowrank_operator -- Sec. 3 eqs. massFinal / stiffnessFinal with the TT
                      cores of eq. TTranks as the canonical terms.
  kron_apply       -- y = sum_a (A_1^a (x) A_2^a (x) A_3^a) x, written out with
                      scipy.sparse.kron (the definition).
  kron_apply_modes -- the same product as three mode products (the Kronecker
                      identity), for large grids.

Pins: TT-SVD reproduces random exact-rank tensors and respects its error
bound, separable tensors come out at rank 1; the univariate route equals the
3-D assembly on exact-rank geometry; kron_apply equals an explicit dense
Kronecker product on tiny sizes, and kron_apply_modes equals kron_apply.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def tt_svd(W, tol, rmax=None, norm=None):
    """TT-SVD of a 3-way array.  Returns cores [(1,n1,r1), (r1,n2,r2), (r2,n3,1)].

    The truncation is relative to `norm` (default ||W||_F).  When the whole
    tensor is below tol * norm it is dropped: the function returns None
    (rank 0).
    """
    W = np.asarray(W, dtype=np.float64)
    n = W.shape
    D = W.ndim
    nrm = np.linalg.norm(W)
    ref = nrm if norm is None else norm
    if nrm <= tol * ref or nrm == 0.0:
        return None
    delta = tol * ref / np.sqrt(D - 1)
    cores = []
    r_prev = 1
    C = W.reshape(r_prev * n[0], -1)
    for d in range(D - 1):
        C = C.reshape(r_prev * n[d], -1)
        U, s, Vt = np.linalg.svd(C, full_matrices=False)
        # smallest rank with tail norm <= delta
        tail = np.sqrt(np.cumsum((s ** 2)[::-1]))[::-1]       # tail[k] = ||s[k:]||
        r = len(s)
        for k in range(1, len(s) + 1):
            if k == len(s) or tail[k] <= delta:
                r = k
                break
        if rmax is not None:
            r = min(r, rmax)
        r = max(r, 1)
        cores.append(U[:, :r].reshape(r_prev, n[d], r))
        C = s[:r, None] * Vt[:r]
        r_prev = r
    cores.append(C.reshape(r_prev, n[-1], 1))
    return cores


def tt_full(cores):
    """Contract TT cores back to the full array."""
    T = cores[0]
    for G in cores[1:]:
        T = np.tensordot(T, G, axes=([-1], [0]))
    return T.reshape(T.shape[1:-1])


def tt_ranks(cores):
    return tuple(c.shape[2] for c in cores[:-1])


def univariate_band(V, D, first, n, w, du_row, du_col):
    """One univariate factor in band form, shape (n, 2p+1).

    A(i, j) = sum_{e,q} w(e,q) phi_i(x_eq) phi_j(x_eq), where phi is the basis
    value or its derivative (du_row for the row index i, du_col for j).
    V, D: local tables (E, q, p+1); first: (E,) first index per element;
    w: (E, q) weight samples (Gauss weights included).
    Returns band[i, o] = A(i, i + o - p).
    """
    E, q, pp1 = V.shape
    p = pp1 - 1
    band = np.zeros((n, 2 * p + 1))
    R = D if du_row else V
    C = D if du_col else V
    for e in range(E):
        loc = np.einsum("x,xa,xb->ab", w[e], R[e], C[e])
        for a in range(pp1):
            for b in range(pp1):
                band[first[e] + a, b - a + p] += loc[a, b]
    return band


def band_dense(band):
    n, nb = band.shape
    p = (nb - 1) // 2
    A = np.zeros((n, n))
    for i in range(n):
        for o in range(nb):
            j = i + o - p
            if 0 <= j < n:
                A[i, j] = band[i, o]
    return A


def lowrank_operator(disc, tt_weights, kind):
    """Kronecker terms of M (kind 'M') or K (kind 'K') from TT weight cores.

    tt_weights: for 'M' the TT cores of omega*g (on the Gauss grid); for 'K'
    a dict {(k,l): cores of q_kl*g} over all 9 (k,l) (symmetric pairs may
    share cores).  Returns a list of terms, each a list of three dense
    (n_d, n_d) matrices (full space, no Dirichlet reduction): the operator
    is sum_terms A_1 (x) A_2 (x) A_3 (eq. massFinal / stiffnessFinal with the
    TT cores expanded as in eq. TTranks).
    """
    def factors(cores, derivs):
        # derivs[d] = (du_row, du_col) for direction d
        r1 = cores[0].shape[2]
        r2 = cores[1].shape[2]
        mats = [[None] * r1, [[None] * r2 for _ in range(r1)], [None] * r2]
        E = disc.E
        for a in range(r1):
            w = cores[0][0, :, a].reshape(E[0], disc.nquad)
            mats[0][a] = band_dense(univariate_band(disc.V[0], disc.D[0], disc.first[0],
                                                    disc.n[0], w, *derivs[0]))
        for a in range(r1):
            for b in range(r2):
                w = cores[1][a, :, b].reshape(E[1], disc.nquad)
                mats[1][a][b] = band_dense(univariate_band(disc.V[1], disc.D[1], disc.first[1],
                                                           disc.n[1], w, *derivs[1]))
        for b in range(r2):
            w = cores[2][b, :, 0].reshape(E[2], disc.nquad)
            mats[2][b] = band_dense(univariate_band(disc.V[2], disc.D[2], disc.first[2],
                                                    disc.n[2], w, *derivs[2]))
        terms = []
        for a in range(r1):
            for b in range(r2):
                terms.append([mats[0][a], mats[1][a][b], mats[2][b]])
        return terms

    if kind == "M":
        return factors(tt_weights, [(False, False)] * 3)
    terms = []
    for (k, l), cores in tt_weights.items():
        if cores is None:
            continue
        # delta(l,d) acts on the row function, delta(k,d) on the column function
        derivs = [(l == d, k == d) for d in range(3)]
        terms += factors(cores, derivs)
    return terms


def restrict_interior(terms):
    return [[A[1:-1, 1:-1] for A in t] for t in terms]


def kron_matrix(terms):
    """Sparse sum_a A_1 (x) A_2 (x) A_3 (definition, kron(A1, kron(A2, A3)))."""
    out = None
    for A1, A2, A3 in terms:
        T = sp.kron(sp.csr_matrix(A1), sp.kron(sp.csr_matrix(A2), sp.csr_matrix(A3)))
        out = T if out is None else out + T
    return out.tocsr()


def kron_apply(terms, x):
    """y = sum_a (A_1^a (x) A_2^a (x) A_3^a) x for x flattened in C order."""
    return kron_matrix(terms) @ np.asarray(x).ravel()


def kron_apply_modes(terms, x):
    """The same y = sum_a (A_1^a (x) A_2^a (x) A_3^a) x through the identity
    (A_1 (x) A_2 (x) A_3) vec(X) = vec(X x_1 A_1 x_2 A_2 x_3 A_3) (three mode
    products on the C-ordered tensor), for grids where the explicit sparse
    Kronecker matrix would be too large."""
    n = tuple(t.shape[1] for t in terms[0])
    X = np.asarray(x, dtype=np.float64).reshape(n)
    out = np.zeros(tuple(t.shape[0] for t in terms[0]))
    for A1, A2, A3 in terms:
        out += np.einsum("ia,jb,kc,abc->ijk", A1, A2, A3, X, optimize=True)
    return out.ravel()


def weight_tts(geo, disc, tol, target=None, samples=None):
    """TT cores of omega*g, q_kl*g (k <= l) and, with a target, yhat*omega*g.

    The weights are sampled on the tensor Gauss grid of the discretisation
    with the quadrature weights folded in.  The entries of Q are truncated
    relative to the Frobenius norm of all of Q, so entries that vanish
    analytically (off-diagonal q_kl of the annulus) drop to rank 0.
    Returns {'omega': cores, (k, l): cores or None, 'load': cores or None}.
    `samples` may pass the output of assemble.sample_weights for this grid
    (to compress one sample at several tolerances).
    """
    from .assemble import sample_weights, evaluate_target
    G, omega, Q, _ = samples if samples is not None else sample_weights(geo, disc)
    _, gs = disc.gauss_grid()
    g = np.einsum("a,b,c->abc", gs[0], gs[1], gs[2])
    out = {"omega": tt_svd(omega * g, tol)}
    qn = np.linalg.norm(Q * g[..., None, None])
    for k in range(3):
        for l in range(k, 3):
            out[(k, l)] = tt_svd(Q[..., k, l] * g, tol, norm=qn)
    if target is not None:
        f = evaluate_target(target, G.reshape(-1, 3)).reshape(omega.shape) * omega * g
        out["load"] = tt_svd(f, tol)
    return out


def lowrank_mk(disc, tts):
    """Kronecker terms of M and K (full space) from weight_tts output."""
    Mterms = lowrank_operator(disc, tts["omega"], "M")
    kl = {}
    for k in range(3):
        for l in range(3):
            kl[(k, l)] = tts[(min(k, l), max(k, l))]
    Kterms = lowrank_operator(disc, kl, "K")
    return Mterms, Kterms


def lowrank_load(disc, cores):
    """Load vector b = sum_t (x)_d b_d[t] from the TT of yhat*omega*g (full space).

    b_d[t](i) = sum_{e,q} f_t(e,q) phi_i(x_eq): the univariate integral of
    the load density against each basis function.
    """
    n = disc.n
    if cores is None:
        return np.zeros(n)
    vecs = []
    for d in range(3):
        C = cores[d]
        r0, Q, r1 = C.shape
        E = disc.E[d]
        v = np.zeros((r0, n[d], r1))
        for a in range(r0):
            for b in range(r1):
                w = C[a, :, b].reshape(E, disc.nquad)
                for e in range(E):
                    v[a, disc.first[d][e]:disc.first[d][e] + disc.degree[d] + 1, b] += \
                        w[e] @ disc.V[d][e]
        vecs.append(v)
    return tt_full(vecs)
