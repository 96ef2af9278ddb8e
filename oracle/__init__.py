"""FP64 CPU oracle for l1 filtering PCP (Liu, Lin, Wei, Su; arXiv 1108.5359).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference legs of ``bench.py`` may import this package.
The library (``paper_1108_5359_gb300``) never imports it and never falls back
to it; the two share no code.  Inputs come from
``paper_1108_5359_gb300.synth`` (input construction only), which the callers
pass in as plain arrays.

Plain, slow, obviously correct NumPy in float64, following the paper's
algorithms in their order and notation:

* ``pcp``      -- soft shrinkage (Section 2), singular value thresholding
                  (Eq. SVT), and the inexact-ALM / ADM solver for PCP
                  (Eq. PCP, Eq. SPCP), used for the seed and, on tiny inputs,
                  for the whole matrix.
* ``l1filter`` -- Algorithm 1 (ADM for the l1 regression Eq. l1g) and
                  Algorithm 2 (the complete l1 filtering method, with the
                  Nystrom representation Eq. l1s').
* ``lp``       -- independent pins for Algorithm 1: exact l1 regression by
                  vertex enumeration, by linear programming, and an
                  optimality (KKT) certificate.

Every function is pinned by ``tests/test_oracle_*.py`` against facts the
paper and the mathematics fix (closed forms, exact recovery, brute force,
LP optima, printed Table 1 norms).  Iteration counts and intermediate ADM
states depend on constants the paper leaves open and are parity unpinned;
only final results are compared.
"""

from . import pcp, l1filter, lp  # noqa: F401
