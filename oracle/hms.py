"""Oracle O2: the hierarchical master-slave iteration, step by step (test infrastructure only).

Follows Secs. 2.1-2.2 and the flowchart of Sec. 3 (Fig. 3) with the readings
listed below; every step is a plain loop or a library primitive (sparse
matrix product, LAPACK banded Cholesky), in FP64, with no fusion.

One iteration, from the current displacement u (u = 0 at the start):

1. r = p - K u on the free DOFs; R1 = ||r||_1 / ||p||_1 (Eq. 19).  Stop when
   R1 < tol.
2. For every set I, from the same u: the displacement-controlled relaxation
   of Eq. 12 with the outer displacements held, written as the increment
   delta_I = u^RD - u^old = (k^Inner_I)^-1 r_I (Eq. 13).  k^Inner_I is K
   restricted to the free DOFs of set I (Eq. 11: "the same components as the
   global matrix"), factored once (end of Sec. 2.2).
3. The q = 9 incremental modes of every set on its free DOFs: translations
   (Eq. 9), constant gradients (Eq. 10), delta and its two gradient-weighted
   copies (Eqs. 13-14), with xi = x - x^(I), eta = y - y^(I).
4. The upper-level matrix K_aa = V^T K V (Eq. 6) and force P = V^T r (Eq. 7).
5. The upper-level system K_aa a = P (Eq. 8), by a Jacobi-scaled Cholesky that
   drops degenerate modes (``coarse_solve``).
6. u <- u + V a (Eq. 3).

Readings (the paper is silent on these):

* the representing node (x^(I), y^(I)) of Eq. 10 is the centroid of the set's
  nodes; the span of the modes, hence the iterate, does not depend on it;
* sets are rectangular node tiles of sx x sy nodes in a row-major set grid,
  the last tile of a row or column takes the remainder;
* q = 9 (the displacement-controlled modes only) by default; ``solve(...,
  force=ForceFactors(...))`` adds the force-controlled modes 10-12 of Eqs.
  15-18 (q = 12; the floating-set reading is in ``ForceFactors``);
* an extended relaxation region (``LocalFactors(overlap=e)``) relaxes the set
  together with a ring of e nodes around it and keeps the set's part of the
  increment as its mode;
* a mode whose diagonal entry of K_aa is <= 1e-300, or <= 1e-28 times the
  largest diagonal entry among its set's nine modes (the mode vanishes on the
  set's free DOFs up to rounding, e.g. eta-modes of a one-row set), or whose
  scaled Cholesky pivot is <= 1e-14 (dependent on earlier modes) gets a = 0,
  in the fixed order (set, mode).
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .direct import to_lower_band
from .truss import BAR_DIRS, Truss, bar_stiffness, bars

NMODES = 9
NMODES_RF = 12  # with the force-controlled modes 10-12 of Eqs. 17-18
DROP_DIAG = 1e-300
DROP_DIAG_REL = 1e-28
DROP_PIVOT = 1e-14


@dataclasses.dataclass
class SetGrid:
    """Rectangular node tiles: set (Ix, Iy) holds nodes i in [Ix*sx, ...),
    j in [Iy*sy, ...); set index I = Iy * Mx + Ix."""
    nx: int
    ny: int
    sx: int
    sy: int

    @property
    def Mx(self):
        return -(-self.nx // self.sx)

    @property
    def My(self):
        return -(-self.ny // self.sy)

    @property
    def M(self):
        return self.Mx * self.My

    def node_set(self):
        """Set index of every node, array [ny, nx]."""
        j, i = np.meshgrid(np.arange(self.ny), np.arange(self.nx), indexing="ij")
        return (j // self.sy) * self.Mx + (i // self.sx)


def rep_points(truss: Truss, grid: SetGrid):
    """Representing node of every set: the centroid of its nodes."""
    ns = grid.node_set().reshape(-1)
    cnt = np.bincount(ns, minlength=grid.M).astype(np.float64)
    xc = np.bincount(ns, weights=truss.x.reshape(-1), minlength=grid.M) / cnt
    yc = np.bincount(ns, weights=truss.y.reshape(-1), minlength=grid.M) / cnt
    return xc, yc


class LocalFactors:
    """k^Inner of every set's relaxation region, factored once (end of Sec. 2.2).

    With ``overlap`` = e > 0 the relaxation region of set I is extended as
    Sec. 2.2 allows (the region drawn around Set_I in Fig. 1): the nodes within
    e nodes of the set's tile in i and in j, clipped to the lattice.  k^Inner is
    then K restricted to the region's free DOFs, every DOF outside the region is
    held, and the mode delta_I of Eq. 13 is the region's increment restricted
    to the set's own DOFs (reading: the sets stay disjoint, so V keeps one block
    of modes per set).  e = 0 is the set itself.
    """

    def __init__(self, truss: Truss, grid: SetGrid, overlap: int = 0, sets=None):
        """``sets``: factor only these set indices (the others relax to 0);
        None = every set."""
        if overlap < 0:
            raise ValueError("overlap must be >= 0")
        self.overlap = overlap
        keep = None if sets is None else set(int(I) for I in sets)
        jn, inode = np.meshgrid(np.arange(grid.ny), np.arange(grid.nx), indexing="ij")
        self.dofs = []     # the set's free DOFs
        self.region = []   # the region's free DOFs (ascending)
        self.pos = []      # where the set's DOFs sit in the region's
        self.factors = []
        K = truss.K.tocsr()
        for I in range(grid.M):
            Ix, Iy = I % grid.Mx, I // grid.Mx
            i0, j0 = Ix * grid.sx, Iy * grid.sy
            i1, j1 = min(grid.nx, i0 + grid.sx), min(grid.ny, j0 + grid.sy)
            in_set = (inode >= i0) & (inode < i1) & (jn >= j0) & (jn < j1)
            e = overlap
            in_reg = (inode >= i0 - e) & (inode < i1 + e) & (jn >= j0 - e) & (jn < j1 + e)
            d = np.flatnonzero(np.repeat(in_set.reshape(-1), 2) & truss.free)
            dr = np.flatnonzero(np.repeat(in_reg.reshape(-1), 2) & truss.free)
            self.dofs.append(d)
            self.region.append(dr)
            self.pos.append(np.searchsorted(dr, d))
            if d.size == 0 or (keep is not None and I not in keep):
                self.factors.append(None)
                continue
            kin = K[dr][:, dr]
            self.factors.append(sla.cholesky_banded(to_lower_band(kin), lower=True))

    def relax(self, r: np.ndarray) -> np.ndarray:
        """delta with delta_I = [(k^Inner_R)^-1 r_R] on set I's DOFs, R its
        relaxation region (Eqs. 12-13; R = I without overlap)."""
        delta = np.zeros_like(r)
        for d, dr, pos, cb in zip(self.dofs, self.region, self.pos, self.factors):
            if cb is not None:
                delta[d] = sla.cho_solve_banded((cb, True), r[dr])[pos]
        return delta


class ForceFactors:
    """Force-controlled relaxation of every set (Eqs. 15-17).

    The set is cut free: Delta k of Eq. 15 adds, on the diagonal block of each
    inner node i, the blocks k_il of K that couple it to nodes l outside the
    set, so k^Inner + Delta k is the stiffness of the set's own bars on its
    free DOFs.  Eq. 16's right-hand side minus (k^Inner + Delta k) u^Inner-old
    is r_I, so the increment of Eq. 17 solves (k^Inner + Delta k) delta^RF = r_I.
    A set clear of the supports floats: the matrix is singular (rigid motions;
    also the mechanisms of one-row or one-column sets) and the paper does not
    say how its solver treated that.  Reading: the minimum-norm solution of the
    system with r_I projected onto the matrix's range, from a dense
    eigendecomposition in which eigenvalues <= ZERO times the largest count as
    zero.
    """
    ZERO = 1e-10

    def __init__(self, truss: Truss, grid: SetGrid):
        ns = grid.node_set().reshape(-1)
        K = truss.K.tocsr()
        a, b, d = bars(truss.nx, truss.ny)
        k = bar_stiffness(truss.nx, truss.ny, truss.ea, truss.L)
        e = BAR_DIRS[d]
        cut = ns[a] != ns[b]
        self.dofs, self.mats, self.eig = [], [], []
        for I in range(grid.M):
            dI = np.flatnonzero((np.repeat(ns, 2) == I) & truss.free)
            loc = {g: q for q, g in enumerate(dI)}
            kf = K[dI][:, dI].toarray()
            # Eq. 15: each cut bar's inner end i gets k_il = -(EA/L) e e^T on its diagonal block
            for t in np.flatnonzero(cut & ((ns[a] == I) | (ns[b] == I))):
                i = a[t] if ns[a[t]] == I else b[t]
                for pp in range(2):
                    for qq in range(2):
                        gp, gq = 2 * i + pp, 2 * i + qq
                        if gp in loc and gq in loc:
                            kf[loc[gp], loc[gq]] -= k[t] * e[t, pp] * e[t, qq]
            w, Q = np.linalg.eigh(kf) if dI.size else (np.zeros(0), np.zeros((0, 0)))
            keep = w > self.ZERO * (w.max() if w.size else 0.0)
            self.dofs.append(dI)
            self.mats.append(kf)
            self.eig.append((w[keep], Q[:, keep]))

    def relax(self, r: np.ndarray) -> np.ndarray:
        """delta^RF with delta^RF_I = (k^Inner_I + Delta k_I)^+ r_I (Eq. 17)."""
        delta = np.zeros_like(r)
        for dI, (w, Q) in zip(self.dofs, self.eig):
            if w.size:
                delta[dI] = Q @ ((Q.T @ r[dI]) / w)
        return delta


def modes(truss: Truss, grid: SetGrid, delta: np.ndarray, rep=None,
          mode_mask: int = 0x1FF, delta_rf: np.ndarray | None = None) -> sp.csc_matrix:
    """Incremental modes V (2N x 9M, column I*9 + m = mode m+1 of set I).

    Eq. 9 (translations), Eq. 10 (constant gradients), Eq. 13 (delta) and
    Eq. 14 (xi*delta, eta*delta); every mode is zero outside its set and on
    constrained DOFs.  Bit m of ``mode_mask`` keeps mode m+1.  With
    ``delta_rf`` (the force-controlled increment of Eq. 17) the modes 10-12
    of Eqs. 17-18 follow: V is 2N x 12M, column I*12 + m.
    """
    xc, yc = rep_points(truss, grid) if rep is None else rep
    ns = grid.node_set().reshape(-1)
    xi = truss.x.reshape(-1) - xc[ns]
    eta = truss.y.reshape(-1) - yc[ns]
    nn = ns.size
    one, zero = np.ones(nn), np.zeros(nn)
    dx, dy = delta[0::2], delta[1::2]
    fields = [  # (x component, y component) per node
        (one, zero), (zero, one),
        (xi, zero), (eta, zero), (zero, xi), (zero, eta),
        (dx, dy), (xi * dx, xi * dy), (eta * dx, eta * dy),
    ]
    nm = NMODES
    if delta_rf is not None:
        fx_, fy_ = delta_rf[0::2], delta_rf[1::2]
        fields += [(fx_, fy_), (xi * fx_, xi * fy_), (eta * fx_, eta * fy_)]
        nm = NMODES_RF
        mode_mask |= 0x7 << NMODES
    free = truss.free
    rows, cols, vals = [], [], []
    node = np.arange(nn)
    for m, (fx, fy) in enumerate(fields):
        if not (mode_mask >> m) & 1:
            continue
        for c, f in ((0, fx), (1, fy)):
            dof = 2 * node + c
            keep = free[dof] & (f != 0)
            rows.append(dof[keep]); cols.append(ns[keep] * nm + m); vals.append(f[keep])
    rows = np.concatenate(rows); cols = np.concatenate(cols); vals = np.concatenate(vals)
    return sp.csc_matrix((vals, (rows, cols)), shape=(truss.ndof, nm * grid.M))


def coarse_system(truss: Truss, V: sp.spmatrix, r: np.ndarray):
    """K_aa = V^T K V (Eq. 6) and P = V^T r (Eq. 7), dense FP64."""
    KV = truss.K @ V
    Kaa = (V.T @ KV).toarray()
    P = V.T @ r
    return Kaa, np.asarray(P).reshape(-1)


def coarse_solve(Kaa: np.ndarray, P: np.ndarray, drop_diag=DROP_DIAG, drop_pivot=DROP_PIVOT,
                 group=NMODES, drop_diag_rel=DROP_DIAG_REL):
    """Solve Eq. 8 by a Jacobi-scaled Cholesky that drops degenerate modes.

    With D = diag(K_aa), the matrix D^-1/2 K_aa D^-1/2 (unit diagonal) is
    factored column by column in index order; a column whose D entry is
    <= drop_diag or <= drop_diag_rel times the largest D of its group (the
    nine modes of one set), or whose pivot is <= drop_pivot, is removed from
    the system (its coefficient is 0).  Returns (a, dropped mask).
    """
    n = P.size
    D = np.diag(Kaa).copy()
    gmax = np.repeat(D.reshape(-1, group).max(axis=1), group) if n % group == 0 else np.full(n, D.max())
    active = (D > drop_diag) & (D > drop_diag_rel * gmax)
    s = np.zeros(n)
    s[active] = 1.0 / np.sqrt(D[active])
    A = s[:, None] * Kaa * s[None, :]
    b = s * P
    L = np.zeros((n, n))
    for m in range(n):
        if not active[m]:
            continue
        v = A[m:, m] - L[m:, :m] @ L[m, :m]
        if v[0] <= drop_pivot:
            active[m] = False
            continue
        d = np.sqrt(v[0])
        L[m, m] = d
        L[m + 1:, m] = v[1:] / d
    y = np.zeros(n)
    for m in range(n):
        if active[m]:
            y[m] = (b[m] - L[m, :m] @ y[:m]) / L[m, m]
    x = np.zeros(n)
    for m in range(n - 1, -1, -1):
        if active[m]:
            x[m] = (y[m] - L[m + 1:, m] @ x[m + 1:]) / L[m, m]
    return s * x, ~active


@dataclasses.dataclass
class Result:
    u: np.ndarray
    history: list          # per residual evaluation: dict(R1, R2, Pi)
    iterations: int        # master updates performed (NIR)
    converged: bool
    iterates: list         # u after each update (if requested)
    dropped: list          # dropped-mode masks per update


def solve(truss: Truss, grid: SetGrid, p: np.ndarray, tol: float, max_iter: int,
          u0=None, rep=None, mode_mask: int = 0x1FF, keep_iterates=False,
          factors: LocalFactors | None = None, force: ForceFactors | None = None) -> Result:
    """The paper's iteration (Fig. 3) from u0 (default 0) until R1 < tol;
    with ``force`` the q = 12 modes (force-controlled relaxation too)."""
    free = truss.free
    p = free * np.asarray(p, dtype=np.float64)
    u = np.zeros(truss.ndof) if u0 is None else free * np.asarray(u0, dtype=np.float64)
    p1 = np.abs(p).sum()
    p2 = np.sqrt(p @ p)
    lf = factors if factors is not None else LocalFactors(truss, grid)
    hist, its, drops = [], [], []
    converged = False
    t = 0
    while True:
        r = truss.residual(p, u)
        R1 = np.abs(r).sum() / p1 if p1 > 0 else 0.0
        hist.append(dict(R1=R1, R2=np.sqrt(r @ r) / p2 if p2 > 0 else 0.0,
                         Pi=-0.5 * (u @ (p + r))))
        if R1 < tol:
            converged = True
            break
        if t >= max_iter:
            break
        delta = lf.relax(r)
        if force is None:
            V = modes(truss, grid, delta, rep, mode_mask)
            Kaa, P = coarse_system(truss, V, r)
            a, dropped = coarse_solve(Kaa, P)
        else:
            V = modes(truss, grid, delta, rep, mode_mask, delta_rf=force.relax(r))
            Kaa, P = coarse_system(truss, V, r)
            a, dropped = coarse_solve(Kaa, P, group=NMODES_RF)
        u = u + V @ a
        drops.append(dropped)
        if keep_iterates:
            its.append(u.copy())
        t += 1
    return Result(u, hist, t, converged, its, drops)


def relax_eq12(truss: Truss, grid: SetGrid, p: np.ndarray, u_old: np.ndarray, I: int):
    """u^Inner-RD of set I by Eq. 12 as printed: k^Inner u^RD = p^Inner -
    k^Outer u^Outer-old (outer = every free DOF outside the set).  Returns the
    set's free DOFs and u^RD on them."""
    ns = np.repeat(grid.node_set().reshape(-1), 2)
    free = truss.free
    inner = np.flatnonzero((ns == I) & free)
    outer = np.flatnonzero((ns != I) & free)
    K = truss.K.tocsr()
    kin = K[inner][:, inner].toarray()
    kout = K[inner][:, outer]
    rhs = np.asarray(p, dtype=np.float64)[inner] - kout @ u_old[outer]
    return inner, np.linalg.solve(kin, rhs)
