"""Planted mistakes: each test plants one plausible error in the oracle (on
the CPU, through monkeypatch) and checks that the pin written for that part
of the oracle fails.  Together they show that the pins are not vacuous: a
transposed operand, a dropped weight, a flipped sign or a swapped Kronecker
order does not pass them."""
import numpy as np
import pytest

import oracle.assemble as oassemble
import oracle.kkt as okkt
import oracle.lowrank as olowrank
import scipy.sparse as sp
import test_oracle_assembly as pins_assembly
import test_oracle_bspline as pins_bspline
import test_oracle_kkt as pins_kkt
import test_oracle_lowrank as pins_lowrank


def test_transposed_metric_fails_the_manufactured_solution(monkeypatch):
    # Q = (J J^T)^{-1} omega instead of (J^T J)^{-1} omega (Sec. 3)
    def wrong(J):
        det = np.linalg.det(J)
        omega = np.abs(det)
        JJt = np.einsum("pab,pcb->pac", J, J)
        return omega, np.linalg.inv(JJt) * omega[:, None, None], det
    monkeypatch.setattr(oassemble, "weights_from_jacobian", wrong)
    with pytest.raises(AssertionError):
        pins_assembly.test_manufactured_poisson_converges("annulus")


def test_dropped_jacobian_determinant_fails_the_volume(monkeypatch):
    # omega = 1 in the mass matrix (the |det J| factor dropped)
    right = oassemble.weights_from_jacobian

    def wrong(J):
        omega, Q, det = right(J)
        return np.ones_like(omega), Q, det
    monkeypatch.setattr(oassemble, "weights_from_jacobian", wrong)
    with pytest.raises(AssertionError):
        pins_assembly.test_volume_and_neumann_kernel("annulus")


def test_flipped_kkt_sign_fails_optimality(monkeypatch):
    # +M instead of -M in the second block row of eq. KKTSystem
    def wrong(M, K, beta):
        return sp.bmat([[M, None, K.T], [None, beta * M, M], [K, -M, None]], format="csc")
    monkeypatch.setattr(okkt, "kkt_matrix", wrong)
    with pytest.raises(AssertionError):
        pins_kkt.test_kkt_solution_is_optimal()


def test_flipped_gradient_sign_fails_finite_differences(monkeypatch):
    # beta M u + M lambda instead of beta M u - M lambda
    def wrong(M, K, b, beta, u):
        y = okkt.state_solve(M, K, u)
        lam = okkt.adjoint_solve(M, K, b, y)
        return beta * (M @ u) + M @ lam, y, lam
    monkeypatch.setattr(pins_kkt, "reduced_gradient", wrong)
    with pytest.raises(AssertionError):
        pins_kkt.test_reduced_gradient_matches_finite_differences()


def test_swapped_kronecker_order_fails_the_definition(monkeypatch):
    # kron(A3, kron(A2, A1)) instead of kron(A1, kron(A2, A3)) on C-ordered x
    def wrong(terms):
        out = None
        for A1, A2, A3 in terms:
            T = sp.kron(sp.csr_matrix(A3), sp.kron(sp.csr_matrix(A2), sp.csr_matrix(A1)))
            out = T if out is None else out + T
        return out.tocsr()
    monkeypatch.setattr(olowrank, "kron_matrix", wrong)
    with pytest.raises(AssertionError):
        pins_lowrank.test_kron_apply_definition_tiny()


def test_negated_derivative_fails_finite_differences(monkeypatch):
    right = pins_bspline.basis_all

    def wrong(knots, p, x, nderiv=1):
        v, dv = right(knots, p, x, nderiv)
        return v, (None if dv is None else -dv)
    monkeypatch.setattr(pins_bspline, "basis_all", wrong)
    p, knots = pins_bspline.KNOTS[1]
    with pytest.raises(AssertionError):
        pins_bspline.test_partition_of_unity_and_fd(p, knots)


def test_threshold_without_sqrt_d_minus_1_fails_the_error_bound(monkeypatch):
    # per-unfolding threshold tol ||W|| instead of tol ||W|| / sqrt(D - 1)
    right = olowrank.tt_svd

    def wrong(W, tol, rmax=None, norm=None):
        return right(W, tol * np.sqrt(np.ndim(W) - 1), rmax, norm)
    monkeypatch.setattr(pins_lowrank, "tt_svd", wrong)
    with pytest.raises(AssertionError):
        pins_lowrank.test_tt_svd_threshold_splits_the_budget()


def test_values_for_derivatives_fail_the_univariate_route(monkeypatch):
    # the row factor always takes basis values, never derivatives
    right = olowrank.univariate_band

    def wrong(V, D, first, n, w, du_row, du_col):
        return right(V, D, first, n, w, False, du_col)
    monkeypatch.setattr(olowrank, "univariate_band", wrong)
    with pytest.raises(AssertionError):
        pins_lowrank.test_univariate_route_exact_on_rank_one_geometry("annulus",
                                                                       pins_lowrank.wl.quarter_annulus())


def test_transposed_jacobian_fails_finite_differences(monkeypatch):
    # J[a][k] = dG_k / dxhat_a instead of dG_a / dxhat_k
    import test_oracle_geometry as pins_geometry
    right = pins_geometry.map_and_jacobian

    def wrong(*args):
        G, J = right(*args)
        return G, np.swapaxes(J, 1, 2)
    monkeypatch.setattr(pins_geometry, "map_and_jacobian", wrong)
    with pytest.raises(AssertionError):
        pins_geometry.test_jacobian_matches_finite_differences(pins_geometry.wl.quarter_annulus())


def test_transposed_left_interface_fails_the_frame_projection(monkeypatch):
    # Phi_L[a]^T instead of Phi_L[a] in the local matvec (Sec. 5, eq. KKT_red)
    import oracle.amen as oamen
    import test_oracle_amen as pins_amen
    right = oamen.local_matvec

    def wrong(PhiL, Ad, PhiR, x):
        return right(np.swapaxes(PhiL, 1, 2), Ad, PhiR, x)
    monkeypatch.setattr(pins_amen, "local_matvec", wrong)
    with pytest.raises(AssertionError):
        pins_amen.test_interfaces_equal_frame_projection(1)


def test_unmapped_gauss_weights_fail_the_span_integrals(monkeypatch):
    # weights not scaled by half the element length (the interval map dropped)
    right = pins_bspline.element_quadrature

    def wrong(knots, q):
        x, g = right(knots, q)
        el = np.diff(np.unique(knots))[:, None]
        return x, g * 2.0 / el
    monkeypatch.setattr(pins_bspline, "element_quadrature", wrong)
    with pytest.raises(AssertionError):
        pins_bspline.test_element_quadrature_integrates_on_spans()


def test_mirrored_row_stencil_fails_the_sampled_rows(monkeypatch):
    # the row stencil read as columns: M(r, r - o) in place of M(r, r + o)
    right = pins_assembly.sampled_rows

    def wrong(geo, disc, rows):
        Mr, Kr = right(geo, disc, rows)
        return Mr[:, ::-1, ::-1, ::-1], Kr[:, ::-1, ::-1, ::-1]
    monkeypatch.setattr(pins_assembly, "sampled_rows", wrong)
    with pytest.raises(AssertionError):
        pins_assembly.test_sampled_rows_equal_band()


def _gauss_variant(width_factor, sign):
    right = oassemble.target_values

    def wrong(kind, params, x):
        if kind != oassemble.TARGET_GAUSS:
            return right(kind, params, x)
        c = np.asarray(params[:3])
        return np.exp(sign * np.sum((x - c) ** 2, axis=1) / (width_factor * params[3]))
    return wrong


@pytest.mark.parametrize("width_factor,sign", [(2.0, -1.0), (1.0, 1.0)])
def test_wrong_gaussian_target_fails_its_pins(monkeypatch, width_factor, sign):
    # exp(-|x - c|^2 / (2 w)) (a variance-style width) or exp(+|x - c|^2 / w)
    # (a dropped minus sign) in the desired state of Sec. 4
    import test_oracle_target as pins_target
    wrong = _gauss_variant(width_factor, sign)
    monkeypatch.setattr(pins_target, "target_values", wrong)
    with pytest.raises(AssertionError):
        pins_target.test_gaussian_target_at_its_centre_and_one_width_away()
    monkeypatch.setattr(oassemble, "target_values", wrong)
    with pytest.raises(AssertionError):
        pins_target.test_load_of_the_gaussian_on_the_unit_cube()
    with pytest.raises(AssertionError):
        pins_target.test_load_of_the_gaussian_on_the_annulus_matches_library_quadrature(0.0)


def test_sine_target_with_a_shifted_phase_fails_its_pins(monkeypatch):
    # prod cos(pi x_k) in place of prod sin(pi x_k)
    import test_oracle_target as pins_target
    right = oassemble.target_values

    def wrong(kind, params, x):
        if kind == oassemble.TARGET_SINPROD:
            return np.prod(np.cos(np.pi * x), axis=1)
        return right(kind, params, x)
    monkeypatch.setattr(pins_target, "target_values", wrong)
    with pytest.raises(AssertionError):
        pins_target.test_sine_product_target_vanishes_on_the_faces_and_peaks_in_the_middle()
    monkeypatch.setattr(oassemble, "target_values", wrong)
    with pytest.raises(AssertionError):
        pins_target.test_load_of_the_sine_product_on_the_unit_cube()


@pytest.mark.parametrize("mistake", ["minus", "no_minv"])
def test_wrong_schur_operator_fails_the_reduced_solve_pin(monkeypatch, mistake):
    # (M - beta K M^{-1} K) or (M + beta K K) in place of the Schur operator
    # of eq. KKTSystem after eliminating u and lambda
    right = okkt.reduced_solve

    def wrong(M_apply, K_apply, Minv_apply, beta, b, **kw):
        if mistake == "minus":
            return right(M_apply, K_apply, Minv_apply, -beta, b, **kw)
        return right(M_apply, K_apply, lambda v: v, beta, b, **kw)
    monkeypatch.setattr(okkt, "reduced_solve", wrong)
    with pytest.raises(AssertionError):
        pins_kkt.test_reduced_cg_equals_direct_solve(oassemble_geo(), 1e-3)


def oassemble_geo():
    from paper_1811_06797_gb300 import workloads as wl
    return wl.quarter_annulus()


def test_interpolation_without_the_collocation_solve_fails_its_pin(monkeypatch):
    # node values taken as the spline coefficients (no solve with Bt, eq.
    # weightEquationSolve): exact only up to degree 1, so the quadratic
    # |det J| of the cubic stretch is no longer reproduced
    import oracle.interp as ointerp
    import test_oracle_interp as pins_interp
    from oracle.bspline import basis_all as ba

    def wrong(knots, pt, xg):
        kt = ointerp.interp_knots(knots, pt)
        E, _ = ba(kt, pt, xg, nderiv=0)
        return E
    monkeypatch.setattr(ointerp, "node_to_gauss", wrong)
    with pytest.raises(AssertionError):
        pins_interp.test_polynomial_weights_are_reproduced_exactly("cubic")


@pytest.mark.parametrize("mistake", ["forward_difference_sign", "untransposed_kk", "tau_dropped"])
def test_wrong_space_time_system_fails_the_time_stepping(monkeypatch, mistake):
    # eq. KKTSystem with KK = I (x) tau K + C (x) M: a +1 below C's diagonal,
    # KK instead of KK^T in the first block row, or I (x) K without tau
    import oracle.parabolic as opar
    import test_oracle_parabolic as pins_par
    if mistake == "forward_difference_sign":
        monkeypatch.setattr(opar, "time_difference", lambda nt: sp.diags(
            [np.ones(nt), np.ones(nt - 1)], [0, -1], shape=(nt, nt), format="csr"))
    elif mistake == "untransposed_kk":
        def wrong(M, K, tau, beta, nt):
            MM, KK = opar.space_time_operators(M, K, tau, nt)
            return sp.bmat([[tau * MM, None, KK], [None, tau * beta * MM, -tau * MM],
                            [KK, -tau * MM, None]], format="csc")
        monkeypatch.setattr(opar, "kkt_matrix_parabolic", wrong)
    else:
        def wrong(M, K, tau, nt):
            I = sp.identity(nt, format="csr")
            return (sp.kron(I, M, format="csr"),
                    sp.kron(I, K, format="csr") + sp.kron(opar.time_difference(nt), M, format="csr"))
        monkeypatch.setattr(opar, "space_time_operators", wrong)
    with pytest.raises(AssertionError):
        pins_par.test_time_stepping_reproduces_the_kkt_solution(4, 0.25, 1e-2)


def test_adjoint_sweep_with_a_flipped_coupling_fails_finite_differences(monkeypatch):
    # M lam_{k+1} entering the backward sweep with the wrong sign
    import oracle.parabolic as opar
    import scipy.sparse.linalg as spla
    import test_oracle_parabolic as pins_par

    def wrong(M, K, tau, b, y):
        lu = spla.splu(sp.csc_matrix(M + tau * K.T))
        lam = np.zeros_like(y)
        nxt = np.zeros(y.shape[1])
        for k in range(y.shape[0] - 1, -1, -1):
            lam[k] = lu.solve(-(M @ nxt) + b[k] - tau * (M @ y[k]))
            nxt = lam[k]
        return lam
    monkeypatch.setattr(opar, "adjoint_stepping", wrong)
    monkeypatch.setattr(pins_par, "reduced_gradient_parabolic", opar.reduced_gradient_parabolic)
    with pytest.raises(AssertionError):
        pins_par.test_reduced_gradient_matches_finite_differences()
