"""Oracle O1: the limit of the iteration by its plain definition (test infrastructure only).

The iteration of the paper converges to the unique solution of Eq. 1 with
SPD K (Sec. 2.1).  This module computes u* = K_ff^-1 p_f directly, two ways:

* ``cholesky_solve``: K on the free DOFs in natural DOF order is a band
  matrix (half-bandwidth 2*nx + 3 for the lattice of ``truss``), factored by
  LAPACK's banded Cholesky (a library primitive) and solved by forward and
  back substitution.  Its band storage grows as nx^2 ny, so it serves lattices
  up to a few hundred nodes across.
* ``sparse_solve``: the same system by a sparse direct factorisation (SuperLU,
  a library primitive) with a fill-reducing minimum-degree ordering of the
  symmetric pattern, so that the 1024 x 1024 lattice (2.1 M DOFs) factors in
  a few GB and minutes.  Pinned against ``cholesky_solve`` and a dense solve.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .truss import Truss


def to_lower_band(A: sp.spmatrix):
    """Lower band storage ab[k, j] = A[j + k, j] of a symmetric sparse matrix."""
    A = sp.coo_matrix(A)
    n = A.shape[0]
    low = A.row >= A.col
    rows, cols, vals = A.row[low], A.col[low], A.data[low]
    bw = int((rows - cols).max()) if rows.size else 0
    ab = np.zeros((bw + 1, n))
    np.add.at(ab, (rows - cols, cols), vals)
    return ab


def cholesky_solve(truss: Truss, p: np.ndarray) -> np.ndarray:
    """u* on all DOFs (zeros on constrained DOFs) by banded Cholesky of K_ff."""
    f = truss.fdofs
    ab = to_lower_band(truss.K_ff())
    cb = sla.cholesky_banded(ab, lower=True)
    u = np.zeros(truss.ndof)
    u[f] = sla.cho_solve_banded((cb, True), np.asarray(p, dtype=np.float64)[f])
    return u


def sparse_solve(truss: Truss, p: np.ndarray) -> np.ndarray:
    """u* on all DOFs (zeros on constrained DOFs) by a sparse direct solve of
    K_ff u_f = p_f (SuperLU, minimum degree on the pattern of K_ff + K_ff^T,
    symmetric mode: diagonal pivots)."""
    f = truss.fdofs
    lu = spla.splu(truss.K_ff().tocsc(), permc_spec="MMD_AT_PLUS_A",
                   options=dict(SymmetricMode=True))
    u = np.zeros(truss.ndof)
    u[f] = lu.solve(np.asarray(p, dtype=np.float64)[f])
    return u
