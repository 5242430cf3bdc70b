"""CPU oracle for the symmetry-adapted FTLM hot path (test infrastructure only).

A plain, slow, obviously-correct FP64 restatement of the paper's method:

* ``group``   — closure of site-permutation generators, conjugacy classes, the
  character table from the class algebra, real irreps from isotypic projectors
  (Section 3), Frobenius-Schur indicators.
* ``sector``  — sector dimensions (Eq. 2 digit sums) and per-irrep block
  dimensions from the character formula (Eq. 13 summed by orbit counting).
* ``basis``   — orbit representatives, stabilizers (Eq. 8), n_Gamma(r) and V_r
  (Eqs. 10-11), block offsets (Eq. 13).
* ``native``  — the C part (``ftlm_oracle.c``): brute-force enumeration and the
  pull-form H·v loop of Eqs. 15-16.
* ``lanczos`` — Philox4x32-10 start vectors, the three-term recurrence, the
  tridiagonal eigensolve (LAPACK) and the thermal sums of Eqs. 4-7, 14.
* ``dense``   — full exact diagonalisation and the explicit projected basis
  vectors of Eq. 12 (the dense projector check of Section 4.1).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it and
shares no code with it.
"""
