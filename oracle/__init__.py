"""Plain FP64 CPU oracle for the low-rank IgA optimal-control path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
product path (the CUDA library and its Python binding) never imports, calls or
links anything here, and this package imports nothing from the product.

Every function restates the paper's definition in the most direct form that
still finishes on small inputs (numpy / scipy primitives as single steps, no
blocking or fusion beyond the definition):

  bspline   -- open knot vectors, Gauss-Legendre rule, Cox-de Boor (Sec. 2)
  geometry  -- NURBS volume map, Jacobian, omega = |det grad G| and
               Q = (J^T J)^{-1} omega (Sec. 2, Sec. 3)
  assemble  -- 3-D tensor-Gauss assembly of M, K and the load vector
               (Sec. 2 eqs. massMatrix / stiffnessMatrix), Dirichlet
               reduction (Sec. 4), sampled rows for large grids
  lowrank   -- TT-SVD (Sec. 3 eq. tt), univariate factors (Sec. 3 eqs.
               massMatrix1D / stiffnessFinal), Kronecker-sum apply
  kkt       -- stationary KKT system (Sec. 4 eq. KKTSystem with N_t = 1),
               direct solve, objective, reduced gradient, and the
               fast-diagonalisation solve on the unit cube
  amen      -- frame matrix (Sec. 5 eq. frame), projected local KKT
               operator (Sec. 5 eq. KKT_red) and its interface form
  interp    -- the weights interpolated in a spline space of degree 2p+1 by
               per-direction collocation (Sec. 3 eqs. weightEquationSystem /
               weightEquationSolve), mapped to the Gauss points
  solve     -- the KKT solve at sizes beyond the direct solve: low-rank
               operators and CG on the reduced system
  parabolic -- the time-dependent KKT system (Sec. 4 eqs. timeDiscrete /
               KKTSystem with N_t steps), direct solve, implicit Euler
               sweeps of the state and the adjoint, objective and reduced
               gradient

Parity status per function is stated in each module header; every function
listed above is pinned by a ``-m "not gpu"`` test against a closed form,
invariant, library routine or brute force, except where a header says
"parity unpinned".
"""
