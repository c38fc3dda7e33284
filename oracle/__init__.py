"""Plain FP64 CPU oracle for the Line-DG hot path (Persson, "A sparse and
high-order accurate line-based discontinuous Galerkin method for unstructured
meshes").

TEST INFRASTRUCTURE ONLY. This package exists to check the CUDA library. Only
the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run it; the library never does, and nothing here
imports the library. It follows the paper's scheme step by step in plain
numpy (vectorised over elements and lines only), in float64 (complex128 for
complex-step derivatives), with M^{-1} applied through a Cholesky
factorisation as the paper prescribes.

Modules and what each follows:
  rules      1-D node set, Gauss-Legendre rule, Lagrange basis, mass matrix
             (Sec. 2.1 Eqs. 8-9, Sec. 2.2)
  mesh       face matching, neighbour nodes, switch function, metric terms
             (Sec. 2.1 Eqs. 2, 4-6; Sec. 2.2; Sec. 3 switch construction)
  physics    Euler/Navier-Stokes/Poisson/advection fluxes, Roe and
             Lax-Friedrichs numerical fluxes (Sec. 5.2 Eqs. 44-48, Sec. 5.1)
  residual   LDG gradient D(U) and residual R(U,Q) (Eqs. 7, 10, 19-32),
             Neumann sides (Eqs. 29-30), the stabilised trace with C22 and
             the coupled split residual (R, Q - D(U, Q)) (Eqs. 26, 36)
  jacobian   K11, K12, K21 and A by complex step (Sec. 4.1 Eq. 35, Eq. 40),
             the coupled Jacobian [[K11, K12], [-K21, I - K22]]
  solvers    split matvec, masked block-Jacobi / ILU(0), GMRES, Newton-BDF2
             (Sec. 4.2 Eqs. 39-41), DIRK3 and RK4 (Sec. 4.1)
  mlp        line-local MLP forward/backward and Adam (not in the paper)

Parity status: every function is pinned by a `-m "not gpu"` test against a
closed form, a library routine, a printed table of the paper, an invariant or
brute force, except the MLP's predictive gain ("parity unpinned": an
empirical claim judged by the FP64 residual).
"""
