"""Oracle: 3-D tensor-Gauss assembly of the mass and stiffness matrices.

Test infrastructure only (see the package header).

Definitions (Sec. 2, eqs. massMatrix and stiffnessMatrix):
  M_ij = int beta_i beta_j omega dxhat,
  K_ij = sum_{k,l} int q_kl  d_l beta_i  d_k beta_j dxhat,
each integral evaluated with the tensor Gauss rule of nquad points per
element and direction, element by element (the standard Galerkin loop).
Dirichlet conditions are imposed by omitting the boundary basis functions
(Sec. 4, discrete QP), i.e. the first and last index in every direction.
Load vector (stationary reading of the right-hand side M yhat of eq.
KKTSystem): b_i = int yhat(G(xhat)) beta_i omega dxhat.

Storage: a "tensor band" array T of shape (n1, n2, n3, 2p1+1, 2p2+1, 2p3+1)
with T[i, o] = A[i, i + o - p]; `band_to_csr` turns it into scipy CSR.

Pins: unit cube M and K equal Kronecker products of closed-form 1-D
matrices; 1^T M 1 is the domain volume; K 1 = 0 without Dirichlet
reduction; symmetry and definiteness; agreement with `dense_bruteforce`
(a separately written per-point loop over full basis vectors) on 4^3
elements; manufactured Poisson solutions converge at rate p+1; the desired
state yhat at points where its definition gives the value outright, and the
load vector summed over the full space against int_Omega yhat dx in closed
form (unit cube) or by library quadrature (annulus, twisted annulus).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .bspline import basis_all, element_quadrature, elements, check_open_knots
from .geometry import map_and_jacobian, weights_from_jacobian, grid_points

TARGET_ZERO, TARGET_SINPROD, TARGET_GAUSS = 0, 1, 2


def target_values(kind, params, x):
    """Desired state yhat at physical points x (P, 3)."""
    if kind == TARGET_ZERO:
        return np.zeros(len(x))
    if kind == TARGET_SINPROD:
        return np.prod(np.sin(np.pi * x), axis=1)
    if kind == TARGET_GAUSS:
        c = np.asarray(params[:3])
        return np.exp(-np.sum((x - c) ** 2, axis=1) / params[3])
    raise ValueError(kind)


def evaluate_target(target, x):
    """A workload target (kind, params) or any callable f(x) at points x (P, 3)."""
    if callable(target):
        return np.asarray(target(x), dtype=np.float64)
    return target_values(target.kind, target.params(), x)


class Discretisation:
    """Per-direction quadrature data of a tensor B-spline space."""

    def __init__(self, degree, knots, nquad):
        self.degree = tuple(int(p) for p in degree)
        self.knots = tuple(np.asarray(k, dtype=np.float64) for k in knots)
        self.nquad = int(nquad)
        self.n = tuple(check_open_knots(k, p) for k, p in zip(self.knots, self.degree))
        self.x, self.g, self.first, self.V, self.D = [], [], [], [], []
        for k, p in zip(self.knots, self.degree):
            x, g = element_quadrature(k, self.nquad)
            el = elements(k)
            # first nonzero basis index on each element: span mu - p
            mu = np.searchsorted(k, el[:, 0], side="right") - 1
            first = mu - p
            v, dv = basis_all(k, p, x.ravel())
            E = len(el)
            idx = first[:, None] + np.arange(p + 1)[None, :]          # (E, p+1)
            V = np.take_along_axis(v.reshape(E, self.nquad, -1), idx[:, None, :], axis=2)
            D = np.take_along_axis(dv.reshape(E, self.nquad, -1), idx[:, None, :], axis=2)
            self.x.append(x)
            self.g.append(g)
            self.first.append(first)
            self.V.append(V)        # (E, q, p+1) local values
            self.D.append(D)        # (E, q, p+1) local derivatives
        self.E = tuple(len(f) for f in self.first)

    def gauss_grid(self):
        """The three 1-D Gauss point sets (flattened E*q) and their weights."""
        return [x.ravel() for x in self.x], [g.ravel() for g in self.g]


def sample_weights(geo, disc):
    """omega, Q on the full tensor Gauss grid, shape (Q1, Q2, Q3[, 3, 3])."""
    xs, _ = disc.gauss_grid()
    pts = grid_points(xs)
    G, J = map_and_jacobian(geo.kind, geo.degree, geo.knots, geo.homogeneous(),
                            geo.twist, pts)
    omega, Q, det = weights_from_jacobian(J)
    shp = tuple(len(x) for x in xs)
    return G.reshape(shp + (3,)), omega.reshape(shp), Q.reshape(shp + (3, 3)), det.reshape(shp)



def assemble_band(geo, disc, target=None, chunk=8):
    """Full M, K (tensor band form) and load vector b, no Dirichlet reduction.

    Loops over elements (batched along the first direction in chunks),
    forms the local (p+1)^3 x (p+1)^3 matrices by the tensor Gauss rule and
    scatters them into the global band array.
    """
    p = disc.degree
    q = disc.nquad
    n = disc.n
    E = disc.E
    Gp, omega, Q, _ = sample_weights(geo, disc)
    xs, gs = disc.gauss_grid()
    gw = np.einsum("a,b,c->abc", gs[0], gs[1], gs[2])
    W = omega * gw                                          # omega * quadrature weight
    if target is not None:
        yh = evaluate_target(target, Gp.reshape(-1, 3)).reshape(W.shape)
    nb = tuple(2 * pp + 1 for pp in p)
    Mb = np.zeros(n + nb)
    Kb = np.zeros(n + nb)
    bvec = np.zeros(n)
    la = [np.arange(pp + 1) for pp in p]
    # local multi-index enumeration (a1, a2, a3) in C order
    A1, A2, A3 = np.meshgrid(la[0], la[1], la[2], indexing="ij")
    A1, A2, A3 = A1.ravel(), A2.ravel(), A3.ravel()
    nloc = len(A1)
    for e1s in range(0, E[0], chunk):
        e1 = np.arange(e1s, min(E[0], e1s + chunk))
        # element grid (e1, e2, e3) and point grid (q, q, q) per element
        V1, D1 = disc.V[0][e1], disc.D[0][e1]          # (c, q, p1+1)
        V2, D2 = disc.V[1], disc.D[1]
        V3, D3 = disc.V[2], disc.D[2]
        # local basis tables phi[e1,e2,e3, q1,q2,q3, a] and gradients
        def outer(X, Y, Z):
            t = np.einsum("ixa,jyb,kzc->ijkxyzabc", X, Y, Z)
            c, e2n, e3n = X.shape[0], Y.shape[0], Z.shape[0]
            return t.reshape(c, e2n, e3n, q ** 3, nloc)
        phi = outer(V1, V2, V3)
        grad = [outer(D1, V2, V3), outer(V1, D2, V3), outer(V1, V2, D3)]
        # point data for these elements, reshaped to (e1, e2, e3, q^3)
        sl = slice(e1[0] * q, (e1[-1] + 1) * q)
        def per_elem(F):
            c = len(e1)
            F = F[sl].reshape(c, q, E[1], q, E[2], q)
            return F.transpose(0, 2, 4, 1, 3, 5).reshape(c, E[1], E[2], q ** 3)
        Wl = per_elem(W)
        Mloc = np.einsum("ijkx,ijkxa,ijkxb->ijkab", Wl, phi, phi, optimize=True)
        Kloc = np.zeros_like(Mloc)
        for kk in range(3):
            for ll in range(3):
                Ql = per_elem(Q[..., kk, ll] * gw)
                # K_ij += q_kl d_l beta_i d_k beta_j  (row i = a, column j = b)
                Kloc += np.einsum("ijkx,ijkxa,ijkxb->ijkab", Ql, grad[ll], grad[kk],
                                  optimize=True)
        if target is not None:
            Fl = per_elem(W * yh)
            bloc = np.einsum("ijkx,ijkxa->ijka", Fl, phi, optimize=True)
        f1 = disc.first[0][e1][:, None, None]
        f2 = disc.first[1][None, :, None]
        f3 = disc.first[2][None, None, :]
        shape3 = (len(e1), E[1], E[2])
        for a in range(nloc):
            i1 = np.broadcast_to(f1 + A1[a], shape3)
            i2 = np.broadcast_to(f2 + A2[a], shape3)
            i3 = np.broadcast_to(f3 + A3[a], shape3)
            if target is not None:
                np.add.at(bvec, (i1, i2, i3), bloc[..., a])
            for b in range(nloc):
                o = (A1[b] - A1[a] + p[0], A2[b] - A2[a] + p[1], A3[b] - A3[a] + p[2])
                np.add.at(Mb, (i1, i2, i3, o[0], o[1], o[2]), Mloc[..., a, b])
                np.add.at(Kb, (i1, i2, i3, o[0], o[1], o[2]), Kloc[..., a, b])
    return Mb, Kb, bvec


def band_to_csr(T, interior=False):
    """Tensor band array -> scipy CSR (optionally Dirichlet-reduced)."""
    n = T.shape[:3]
    nb = T.shape[3:]
    p = tuple((b - 1) // 2 for b in nb)
    I = np.indices(n + nb).reshape(6, -1)
    vals = T.reshape(-1)
    j = [I[d] + I[3 + d] - p[d] for d in range(3)]
    ok = np.ones(vals.shape, bool)
    for d in range(3):
        ok &= (j[d] >= 0) & (j[d] < n[d])
    if interior:
        lo = 1
        hi = [nn - 1 for nn in n]
        for d in range(3):
            ok &= (I[d] >= lo) & (I[d] < hi[d]) & (j[d] >= lo) & (j[d] < hi[d])
        nn = tuple(x - 2 for x in n)
        off = 1
    else:
        nn = n
        off = 0
    rows = np.ravel_multi_index(tuple(I[d][ok] - off for d in range(3)), nn)
    cols = np.ravel_multi_index(tuple(j[d][ok] - off for d in range(3)), nn)
    N = int(np.prod(nn))
    return sp.csr_matrix((vals[ok], (rows, cols)), shape=(N, N))


def interior_vector(v):
    """Drop the boundary coefficients of a (n1, n2, n3) tensor (Sec. 4)."""
    return v[1:-1, 1:-1, 1:-1]


def dense_bruteforce(geo, disc, target=None):
    """Dense M, K, b by a per-point loop over full basis vectors.

    A second, separately written route to eqs. massMatrix / stiffnessMatrix
    for tiny grids: at every tensor Gauss point evaluate all prod_d n_d
    basis functions and their parametric gradients and accumulate the outer
    products directly (no element bookkeeping, no band storage).
    """
    xs, gs = disc.gauss_grid()
    vals, ders = [], []
    for d in range(3):
        v, dv = basis_all(disc.knots[d], disc.degree[d], xs[d])
        vals.append(v)
        ders.append(dv)
    Gp, omega, Q, _ = sample_weights(geo, disc)
    N = int(np.prod(disc.n))
    M = np.zeros((N, N))
    K = np.zeros((N, N))
    b = np.zeros(N)
    for a in range(len(xs[0])):
        for c in range(len(xs[1])):
            for e in range(len(xs[2])):
                g = gs[0][a] * gs[1][c] * gs[2][e]
                B = np.kron(vals[0][a], np.kron(vals[1][c], vals[2][e]))
                dB = np.stack([
                    np.kron(ders[0][a], np.kron(vals[1][c], vals[2][e])),
                    np.kron(vals[0][a], np.kron(ders[1][c], vals[2][e])),
                    np.kron(vals[0][a], np.kron(vals[1][c], ders[2][e])),
                ])
                w = omega[a, c, e] * g
                M += w * np.outer(B, B)
                # (Q grad beta_i) . grad beta_j  ->  dB^T Q dB  with Q applied on the row side
                K += g * (dB.T @ Q[a, c, e].T @ dB)
                if target is not None:
                    yh = evaluate_target(target, Gp[a, c, e][None, :])[0]
                    b += w * yh * B
    return M, K, b


def sampled_rows(geo, disc, rows):
    """Entries of M and K in the given rows, by the definition.

    rows: (S, 3) integer multi-indices into the full (non-reduced) space.
    Returns (Mrows, Krows) of shape (S, 2p1+1, 2p2+1, 2p3+1) with
    [s, o] = A[rows[s], rows[s] + o - p]; entries outside the index range
    are zero.  Each row is integrated over the elements in the support of
    its basis function only.
    """
    p = disc.degree
    q = disc.nquad
    rows = np.asarray(rows, dtype=np.int64)
    nb = tuple(2 * pp + 1 for pp in p)
    Mr = np.zeros((len(rows),) + nb)
    Kr = np.zeros((len(rows),) + nb)
    hw = geo.homogeneous()
    for s, r in enumerate(rows):
        # elements whose local functions include index r_d
        els = []
        for d in range(3):
            f = disc.first[d]
            els.append(np.nonzero((f <= r[d]) & (r[d] <= f + p[d]))[0])
        for e1 in els[0]:
            for e2 in els[1]:
                for e3 in els[2]:
                    x1, x2, x3 = disc.x[0][e1], disc.x[1][e2], disc.x[2][e3]
                    g = np.einsum("a,b,c->abc", disc.g[0][e1], disc.g[1][e2], disc.g[2][e3]).ravel()
                    pts = grid_points([x1, x2, x3])
                    _, J = map_and_jacobian(geo.kind, geo.degree, geo.knots, hw, geo.twist, pts)
                    omega, Q, _ = weights_from_jacobian(J)
                    V = [disc.V[0][e1], disc.V[1][e2], disc.V[2][e3]]
                    D = [disc.D[0][e1], disc.D[1][e2], disc.D[2][e3]]
                    fs = [disc.first[0][e1], disc.first[1][e2], disc.first[2][e3]]
                    la = [r[d] - fs[d] for d in range(3)]
                    # row function value / gradient at the points
                    vi = np.einsum("a,b,c->abc", V[0][:, la[0]], V[1][:, la[1]], V[2][:, la[2]]).ravel()
                    gi = np.stack([
                        np.einsum("a,b,c->abc", D[0][:, la[0]], V[1][:, la[1]], V[2][:, la[2]]).ravel(),
                        np.einsum("a,b,c->abc", V[0][:, la[0]], D[1][:, la[1]], V[2][:, la[2]]).ravel(),
                        np.einsum("a,b,c->abc", V[0][:, la[0]], V[1][:, la[1]], D[2][:, la[2]]).ravel(),
                    ])                                              # (3, P)
                    for b1 in range(p[0] + 1):
                        for b2 in range(p[1] + 1):
                            for b3 in range(p[2] + 1):
                                vj = np.einsum("a,b,c->abc", V[0][:, b1], V[1][:, b2], V[2][:, b3]).ravel()
                                gj = np.stack([
                                    np.einsum("a,b,c->abc", D[0][:, b1], V[1][:, b2], V[2][:, b3]).ravel(),
                                    np.einsum("a,b,c->abc", V[0][:, b1], D[1][:, b2], V[2][:, b3]).ravel(),
                                    np.einsum("a,b,c->abc", V[0][:, b1], V[1][:, b2], D[2][:, b3]).ravel(),
                                ])
                                o = (fs[0] + b1 - r[0] + p[0], fs[1] + b2 - r[1] + p[1],
                                     fs[2] + b3 - r[2] + p[2])
                                Mr[s, o[0], o[1], o[2]] += np.sum(g * omega * vi * vj)
                                # sum_kl q_kl d_l beta_i d_k beta_j
                                Kr[s, o[0], o[1], o[2]] += np.sum(
                                    g * np.einsum("pkl,lp,kp->p", Q, gi, gj))
    return Mr, Kr


def sampled_load(geo, disc, target, rows):
    """Load entries b_i = int yhat(G) beta_i omega for sampled multi-indices (full space).

    Integrates over the elements in the support of each basis function only,
    with the same tensor Gauss rule as `assemble_band`.
    """
    p = disc.degree
    rows = np.asarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    hw = geo.homogeneous()
    for s, r in enumerate(rows):
        els = []
        for d in range(3):
            f = disc.first[d]
            els.append(np.nonzero((f <= r[d]) & (r[d] <= f + p[d]))[0])
        for e1 in els[0]:
            for e2 in els[1]:
                for e3 in els[2]:
                    pts = grid_points([disc.x[0][e1], disc.x[1][e2], disc.x[2][e3]])
                    g = np.einsum("a,b,c->abc", disc.g[0][e1], disc.g[1][e2], disc.g[2][e3]).ravel()
                    Gp, J = map_and_jacobian(geo.kind, geo.degree, geo.knots, hw, geo.twist, pts)
                    omega, _, _ = weights_from_jacobian(J)
                    yh = evaluate_target(target, Gp)
                    la = [r[0] - disc.first[0][e1], r[1] - disc.first[1][e2], r[2] - disc.first[2][e3]]
                    vi = np.einsum("a,b,c->abc", disc.V[0][e1][:, la[0]], disc.V[1][e2][:, la[1]],
                                   disc.V[2][e3][:, la[2]]).ravel()
                    out[s] += np.sum(g * omega * yh * vi)
    return out
