"""FP64 CPU oracle for the overlap Dirac operator hot path (arXiv:1510.06897).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
library under ``paper_1510_06897_gb300`` never imports it, and this package
never imports the library: the two share no code.  Inputs come from
``paper_1510_06897_gb300.inputs`` (seeded generators only) and are passed in
as arrays.

Everything here is plain, slow NumPy in complex128, written so that a reader
can check it against the paper by eye:

  wilson     D_W (Eq. 2), K = gamma5 (D_W - m_W) (Sec. 2), gamma matrices
  chebyshev  Chebyshev coefficients of y^{-1/2} and the forward three-term
             recurrence that evaluates the polynomial approximation (Eq. 3)
  overlap    deflation, sign(K) in projected and literal form (Eq. 3),
             D[mu] and D[mu]^dagger (Eq. 1)
  cg         textbook conjugate gradient on D^dagger D
  sumr       shifted-unitary minimal residual (SUMR) for D[mu] and the GMRESR
             (GCR) outer loop around a relaxed inner SUMR (Sec. 2)
  smear      over-improved stout smearing of the links (Sec. 3 input preparation)
  dense      dense matrices of D_W / K on tiny lattices and the exact
             sign(K) = V sign(Lambda) V^dagger
  force      gradient of chi^dagger P(K) chi with respect to the links
             (reverse sweep of the forward recurrence) and its forward-mode
             tangent along an su(3) direction

Parity status of each function is listed in its module docstring; all of
them are pinned by tests in ``tests/test_oracle_*.py`` against closed forms,
dense linear algebra, invariants or finite differences.
"""
from . import wilson, chebyshev, overlap, cg, dense, force, sumr, smear  # noqa: F401
