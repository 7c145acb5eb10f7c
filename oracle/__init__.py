"""CPU oracle for the all-at-once Uzawa multigrid Stokes solver -- TEST INFRASTRUCTURE ONLY.

This package is the plain, slow, obviously-correct reference that the CUDA
path is checked against.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it; the product path
(``paper_1511_02134_gb300``) never does, and the two share no code.  The only
shared module is ``workloads`` (seeded inputs, no solver arithmetic).

Everything is float64 numpy/scipy.  Matrices are assembled from element
integrals over an explicitly refined mesh; nothing here uses the lattice
stencils of the CUDA path.

Modules and the passages they follow (paper: Gmeiner, Huber, John, Ruede,
Wohlmuth, arXiv:1511.02134):
  mesh       uniform refinement of the macro mesh (Sec. 2.1, Sec. 4)
  fem        element integrals of a_1, b, c_l, f, g_l (Sec. 2.1)
  stokes     block system K = [A B^T; B -C], Dirichlet elimination, residual (Sec. 3)
  krylov     CG and block-preconditioned MINRES of the coarse grid (Sec. 3.2, 3.7)
  multigrid  inexact Uzawa smoother, V_var(3,3) cycle, stopping rule (Sec. 3.3-3.6)
  direct     exact discrete solution by a sparse direct solve
  adjoint    outflow functional and its gradient w.r.t. the body force
  analysis   operator-count and memory models (Sec. 4.1, 4.2)

Parity pins (tests/test_oracle_*.py) tie each module to something other than
itself: closed-form lattice stencils, consistency invariants, Galerkin
identities of nested spaces, scipy's CG/MINRES, brute-force sequential
Gauss-Seidel, the direct solve, the O(h^2) velocity error of the manufactured
solution, and numbers the paper prints.  Parity unpinned: the paper's exact
iteration counts and times for its hybrid HHG smoother ordering (the ordering
used here is a stated reading), and the paper's own coarse-solver internals.
"""
