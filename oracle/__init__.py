"""CPU oracle for the forward-error-oriented eigenvector refinement (Terao & Ozaki).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package; the
library's product path never does.

It is a plain, slow, independent restatement of the paper in numpy:

* ``ddarith``  -- TwoSum, pair arithmetic (Sec. 2.2) and double-double helpers.
* ``ozaki``    -- the error-free splitting of Sec. 2.3 (eq. sigma, tau, a, x) on a
  fixed 8-bit digit grid, exact integer slice products, recombination.
* ``refine``   -- Algorithm 1 with the Sec. 3 modification (X <- X^(1), n_A-slice
  accurate product) and the Sec. 4.1 choice of alpha and beta; stopping test.
* ``truth``    -- reference eigenvectors of a stored matrix by double-double
  Ogita-Aishima refinement, and the forward-error metric.

Floating point is FP64 and double-double; slice products are exact int64.
Parity pins: every function is pinned by ``tests/test_oracle_*.py`` against
closed forms, brute force, invariants or values worked out by hand from the paper.
Functions without such a pin say "parity unpinned" in their docstring.
"""
