"""Plain FP64 CPU oracle for the block-domain Helmholtz-Poisson solver.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports this package:
only `tests/`, `__graft_entry__.smoke()` and the `cpu_baseline` / reference leg
of `bench.py` may use it.  It shares no code with the CUDA library (the two do
not import each other); the only common module is `workloads`, which makes the
seeded inputs and holds none of the method's arithmetic.

What it computes, each piece by its plain definition:
  geometry  -- the unknowns of a domain: the grid points strictly inside the
               union of the blocks (Sec. 2.3, Fig. "concat"; the cross of Sec. 3)
  operator  -- the global 5-point matrix K of  lap p + kappa p = f  (Eq. 1,
               Eq. "Poisson_central", Eq. "mat_Poisson") with zero Dirichlet data
  direct    -- p = K^{-1} b (dense LU for tiny grids, sparse LU otherwise), and
               conjugate gradients on -K as a second, hand-written route
  transforms-- the DST-I matrix and the closed-form eigenvalues (Eqs.
               "Poisson_spectral_eigen", "eigvector_Diri")
  schur     -- the block pieces A_i, R_ij read off K, the Schur complement
               L_c = A_c - sum_a R_ca A_a^{-1} R_ac and Algorithm 1
               (Eqs. "block_global", "Schur_subeq", Alg. "fft_dd_solver")
  krylov    -- restarted GMRES / flexible GMRES with modified Gram-Schmidt
               Arnoldi and Givens least squares (Sec. 2.4)
  neumann   -- the Neumann line operator, its DCT-II eigenbasis and the Neumann
               rectangle (Sec. 2.2, Eq. "submat_Neumann")
  neumann_cross -- the cross with Neumann arm sides and its analytic solution
               (Sec. 3.1, Eqs. "cross_equation"-"cross_ana_sol_psi")
  periodic  -- the circulant line operator, its real (Hartley) eigenbasis and
               the periodic rectangle (Sec. 2.2, Eq. "submat_Periodic")
  box       -- the 7-point operator of a 3-D box (the 3-D extension after Sec. 2.1)
  strip     -- the chain of crosses, several coupled blocks (Sec. 2.3-2.4)

Parity status: every function above is pinned by `tests/test_oracle_*.py`
(closed forms, brute force on tiny grids, second-order convergence, library
routines, an independent second route: library transforms with banded solves,
conjugate gradients, least squares over the explicit Krylov space).  Iteration counts are "parity unpinned": the paper's plots of them
are lost, only their trend is stated.
"""
