"""Plain complex128 CPU oracle for the EigT/PFFT-preconditioned GMRES Helmholtz solver.

This package is TEST INFRASTRUCTURE. It restates, slowly and in the paper's notation, what the
GPU library computes, so that the CUDA path can be checked element by element.  Only the test
suite (``tests/``), ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it.  The product path never routes through it and it shares no
code with the CUDA library: no kernels, tables, constants or pre/post-processing.

Paper: Gryazin, Gonzales, Li, "High-Resolution Solvers for 3D Helmholtz Scattering Problems Using
PFFT and Eigenvector-Based Preconditioning" (arXiv 2602.07711).

Module map (each function cites the passage it follows):
  grid        grid steps, staggered / collocated nodes, Sommerfeld ghost coefficient (Sec. 2.1, Eq. D_bc)
  operators   A for the 2nd/4th/6th-order compact schemes with ghost elimination (Eqs. scheme4, scheme6)
  rhs         modified right-hand sides f^(IV), f^(VI) (Eqs. scheme4, scheme6)
  eig1d       the 1D ABC matrix Lambda-bar and its eigendecomposition (Eq. lambda_mat_definition)
  tridiag     Thomas algorithm for the z-systems (Eq. Indep_precond_system)
  eigt        EigT direct solver of A_p U = Y (Sec. 4.1, Eq. EIG_SOLVER)
  pfft        PFFT three-step solver (Sec. 4.2, Eq. PFFT_SOLVER)
  gmres       restarted right-preconditioned GMRES(m) and flexible GMRES (Sec. 5, [Saad])
  metrics     L2-err, max-err (Sec. 5.1)
  model1d     the 1D model problem of Sec. 3 (Eqs. vect_eq, coef_gen, precond)
  manufactured  the separable test solution of Sec. 5.1
  closure     high-order ABC closure on collocated grids for the manufactured tests (reading of Sec. 2.1)

Parity status: every function is pinned by a ``-m "not gpu"`` test in tests/test_oracle_*.py.
"""
