"""CPU oracle for the hierarchical master-slave solver -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 NumPy/SciPy code that states what the GPU path must compute,
written from the paper (Xu, Liu, Dong, "Scalable hierarchical parallel
algorithm for the solution of super large-scale sparse linear equations").
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it.  It shares no code with the CUDA library and never
imports it; the product path must not call anything in here.

Parts:

* ``truss``  -- the 2-D triangle-lattice truss of Sec. 3.1: node coordinates,
  bars, the assembled stiffness K of Eq. 1, the residual and the energy of Eq. 2.
* ``direct`` -- O1, the plain definition of the limit: u* = K^-1 p by a direct
  banded Cholesky factorisation of K on the free DOFs.
* ``hms``    -- O2, the paper's iteration step by step: residual, local
  displacement-controlled relaxation (Eqs. 11-14), incremental modes
  (Eqs. 9, 10, 13, 14), the upper-level system (Eqs. 5-8) and the update (Eq. 3),
  stopped by the 1-norm relative residual of Eq. 19.
* ``pool``   -- the same per-set relaxation spread over host processes (the
  sets relax independently), for timing the oracle on all host cores.

Parity status: every function is pinned by the not-gpu tests in
``tests/test_oracle_*.py`` (dense brute force, closed forms, invariants).  The
iteration counts the paper plots (Figs. 5-7) are lost from the text, so the
number of iterations is "parity unpinned" against the paper; it is pinned only
by the invariants of the method (energy decrease, Galerkin orthogonality,
one-set convergence in one step).
"""
from . import truss, direct, hms, pool  # noqa: F401
