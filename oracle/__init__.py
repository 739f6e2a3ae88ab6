"""FP64 CPU oracle for the matrix-free tetrahedral Laplace operators (arxiv 2509.10226).

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of what the GPU library computes.  Only the test suite, the smoke
check in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import
it; the library under ``paper_2509_10226_gb300`` never does, and this package
never imports the library.  The two share no code: this side builds its own
Grundmann-Moeller rule (exact rationals), its own Lagrange basis (monomial
Vandermonde solve), its own DoF numbering (sorted vertex-multiset keys), its own
face matching and evaluates the faces of the DG operator by inverting each
cell's affine map instead of using permutation tables.

Modules
  quadrature  Grundmann-Moeller simplex rules (rule family taken from the
              configurations; the paper names its own rules in Sec. 2.3)
  basis       Lagrange P_p on equispaced nodes (Sec. 2.2, Eq. 4 tables)
  topology    canonical DoF keys, faces, Dirichlet set
  cg          continuous operator, Eq. 3 (apply, adjoint, coefficient gradient,
              diagonal, right-hand side)
  dg          SIPG operator, Eq. 2 and Eq. 5
  solve       plain Jacobi-preconditioned CG in FP64

Every public function is pinned by a ``-m "not gpu"`` test against closed
forms, exact rational integrals or brute force (tests/test_oracle_*.py).  The
one quantity whose value the paper fixes but does not print (its own
Witherden-Vincent / Xiao-Gimbutas rules) is not reproduced: parity unpinned for
that rule family, which no configuration uses.
"""
