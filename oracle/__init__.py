"""Plain FP64 CPU oracle for the pseudo-inverse-preconditioned Wiener solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports, calls or links anything in this package.  Only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.

It restates, in slow and readable NumPy, what the paper (Seljebotn et al.,
arXiv:1710.00621) defines:

* ``grids``    -- Gauss-Legendre and HEALPix ring grids and their quadrature
                  weights (Sec. 2.1, Sec. 2.2, App. A.1).
* ``legendre`` -- normalised associated Legendre functions by the three-term
                  recurrence, with exponent scaling against FP64 underflow.
* ``alm``      -- the real harmonic coefficient layout used at the boundary.
* ``sht``      -- synthesis Y, adjoint synthesis Y^T and analysis Y^T W
                  (Sec. 2.1, Sec. 3.2), ring-factored and as a dense matrix.
* ``model``    -- the data model d = P s + n, P = Y B Q~ (Eqs. block-data-model,
                  P, Q), the system A = S^-1 + P^T N^-1 P (Eq. A) and its RHS.
* ``precond``  -- alpha (Eq. optimal-alpha), q (Eq. optimal-q), the per-l
                  blocks of U (Eqs. U-data, U-prior), U^+ and
                  M_PI = U^+ T^+ (U^+)^T (Eq. fullmodel-preconditioner).
* ``cg``       -- textbook preconditioned conjugate gradients (Sec. 2.3).
* ``closed_form`` -- the per-l diagonal Wiener filter that holds when the
                  inverse-noise map is flat per unit area (Sec. 3.3).

Every function is in FP64 and follows the paper's notation.  Parity status of
each part is listed in the module headers; all parts are pinned by tests in
``tests/test_oracle_*.py`` against closed forms, library routines of other
provenance (scipy spherical harmonics, numpy polynomial quadrature) and
invariants fixed by the paper.
"""
