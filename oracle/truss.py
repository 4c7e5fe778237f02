"""Oracle: the 2-D triangle-lattice truss of Sec. 3.1 (test infrastructure only).

The paper's test problems are square triangle-lattice trusses whose nodes are
joined to their neighbours by elastic rods and loaded by random nodal forces
(Sec. 3.1, Fig. 4).  The figure is lost, so this module states the readings it
uses:

* nodes (i, j), 0 <= i < nx, 0 <= j < ny, in offset rows:
  x = L (i + (j mod 2)/2), y = L j sqrt(3)/2;
* every node owns up to three bars: E to (i+1, j); NE and NW to the two nodes
  of row j+1 at x +- L/2 (for even j these are (i, j+1) and (i-1, j+1), for odd
  j they are (i+1, j+1) and (i, j+1));
* a bar is a linear two-node rod with axial stiffness EA/L, so its element
  stiffness is (EA/L) [[e e^T, -e e^T], [-e e^T, e e^T]] with e the unit
  vector along the bar;
* DOF index of node n = j*nx + i is 2n (x) and 2n + 1 (y).

K assembled from these bars is the matrix of Eq. 1 (symmetric; positive
definite on the free DOFs once rigid motions are removed by supports).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

SQ3_2 = math.sqrt(3.0) / 2.0

# unit vectors of the three owned bar directions (E, NE, NW)
BAR_DIRS = np.array([[1.0, 0.0], [0.5, SQ3_2], [-0.5, SQ3_2]])


def node_xy(nx: int, ny: int, L: float = 1.0):
    """Coordinates x[j, i], y[j, i] of the offset-row triangle lattice."""
    j, i = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    x = L * (i + 0.5 * (j % 2))
    y = L * SQ3_2 * j
    return x.astype(np.float64), y.astype(np.float64)


def bars(nx: int, ny: int):
    """All bars of the lattice as (a, b, d): node a owns the bar of direction d
    (0 = E, 1 = NE, 2 = NW) whose other end is node b."""
    a_list, b_list, d_list = [], [], []
    for j in range(ny):
        for i in range(nx):
            a = j * nx + i
            if i + 1 < nx:
                a_list.append(a); b_list.append(a + 1); d_list.append(0)
            if j + 1 < ny:
                if j % 2 == 0:
                    ne, nw = (i, j + 1), (i - 1, j + 1)
                else:
                    ne, nw = (i + 1, j + 1), (i, j + 1)
                for d, (ii, jj) in ((1, ne), (2, nw)):
                    if 0 <= ii < nx:
                        a_list.append(a); b_list.append(jj * nx + ii); d_list.append(d)
    return (np.array(a_list, dtype=np.int64), np.array(b_list, dtype=np.int64),
            np.array(d_list, dtype=np.int64))


def bar_stiffness(nx: int, ny: int, ea, L: float = 1.0):
    """Axial stiffness EA/L of every bar, in the order of ``bars``.

    ``ea`` is None (EA = 1), a scalar, or an array [3, ny, nx] indexed by the
    owning node and the direction.
    """
    a, _, d = bars(nx, ny)
    if ea is None:
        return np.full(a.shape, 1.0 / L)
    ea = np.asarray(ea, dtype=np.float64)
    if ea.ndim == 0:
        return np.full(a.shape, float(ea) / L)
    jj, ii = np.divmod(a, nx)
    return ea[d, jj, ii] / L


def assemble_K(nx: int, ny: int, ea=None, L: float = 1.0) -> sp.csr_matrix:
    """Global stiffness K (2N x 2N, all DOFs, no supports) summed bar by bar."""
    a, b, d = bars(nx, ny)
    k = bar_stiffness(nx, ny, ea, L)
    e = BAR_DIRS[d]
    rows, cols, vals = [], [], []
    for p in range(2):
        for q in range(2):
            kee = k * e[:, p] * e[:, q]
            for (n1, n2, s) in ((a, a, 1.0), (b, b, 1.0), (a, b, -1.0), (b, a, -1.0)):
                rows.append(2 * n1 + p); cols.append(2 * n2 + q); vals.append(s * kee)
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    n = 2 * nx * ny
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def free_mask(nx: int, ny: int, fixed=None) -> np.ndarray:
    """Boolean vector over the 2N DOFs, True where the DOF is free.

    ``fixed`` is None (bottom row clamped) or a uint8 array [ny, nx, 2]
    with 1 on constrained DOFs.
    """
    if fixed is None:
        fixed = np.zeros((ny, nx, 2), dtype=np.uint8)
        fixed[0] = 1
    return np.asarray(fixed).reshape(-1) == 0


class Truss:
    """Lattice, supports and stiffness of one problem (Eq. 1 with supports).

    Displacement and force vectors are full-length (2N) with zeros on the
    constrained DOFs; K_ff = K restricted to the free DOFs is the SPD system
    matrix.
    """

    def __init__(self, nx, ny, ea=None, fixed=None, L=1.0):
        self.nx, self.ny, self.L = nx, ny, L
        self.ea = ea
        self.K = assemble_K(nx, ny, ea, L)
        self.free = free_mask(nx, ny, fixed)
        self.fdofs = np.flatnonzero(self.free)
        self.x, self.y = node_xy(nx, ny, L)

    @property
    def ndof(self):
        return 2 * self.nx * self.ny

    def K_ff(self) -> sp.csr_matrix:
        f = self.fdofs
        return self.K[f][:, f].tocsr()

    def apply_K(self, u):
        """(K u) on the free DOFs, 0 on constrained DOFs; u is zero there."""
        return self.free * (self.K @ (self.free * u))

    def residual(self, p, u):
        """r = p - K u on the free DOFs (Eq. 7's bracket, Eq. 19's vector)."""
        return self.free * (p - self.K @ (self.free * u))

    def energy(self, p, u):
        """Total energy Pi = 1/2 u.K.u - u.p of Eq. 2 over the free DOFs."""
        uf = self.free * u
        return 0.5 * uf @ (self.K @ uf) - uf @ (self.free * p)

    def reactions(self, u):
        """Forces K u at every DOF, including the constrained ones."""
        return self.K @ (self.free * u)


def flat_loads(p3) -> np.ndarray:
    """Loads [ny, nx, 2] as a 2N vector in DOF order."""
    return np.asarray(p3, dtype=np.float64).reshape(-1)
