"""Serial FP64 CPU oracle for the two-level ORAS-FGMRES Helmholtz solver.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
(the CUDA library and its Python binding) never imports, links or runs it,
and this package imports nothing from the product: the two share only the
seeded input generators in ``synth``.

It is a plain, slow, obviously-correct restatement of the method of
Dolean, Jolivet, Tournier & Operto (EAGE 2020, arXiv 2004.06309):

* ``fem``    -- Eq. (1)-(2): P1/P2 Lagrange assembly of the Helmholtz
  operator with first-order absorbing faces and a Dirichlet top.
* ``dd``     -- Eq. (4): overlapping subdomains, Boolean restrictions R_i,
  partition of unity D_i, local matrices A_i with absorbing (Robin)
  interface conditions.
* ``coarse`` -- Eq. (3): interpolation Z from the coarse mesh, E = Z^T A Z.
* ``krylov`` -- restarted right-preconditioned FGMRES(m) with CGS2 and
  complex Givens rotations; the stopping rule is the relative residual.
* ``solver`` -- the one- and two-level ORAS preconditioner and the solve.

Every function is in FP64 (complex128).  Parity of each part is pinned in
``tests/test_oracle_*.py`` against closed forms, brute force and invariants.
"""
