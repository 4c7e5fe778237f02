"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here touches the GPU.  Each test checks the oracle against something
other than itself: published known answers, a brute-force restatement built
from node coordinates alone, closed forms (rigid modes, the patch test,
equilibrium), textbook special cases (one set = direct solve) and invariants of
the method (energy decrease of Eq. 2, Galerkin orthogonality of Eq. 5,
independence of the representing node of Eq. 10).
"""
import math
import os

import numpy as np
import pytest

from oracle import direct, hms, truss
from workloads import clamp_bottom, ea_lognormal, loads, philox4x32_10

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ3 = math.sqrt(3.0)


# ---------------------------------------------------------------- generators
def test_philox_known_answers():
    """Philox4x32-10 reproduces the Random123 known-answer vectors (SC'11)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip()
            and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        ctr = [int(x, 16) for x in r[0:4]]
        key = [int(x, 16) for x in r[4:6]]
        out = [int(x, 16) for x in r[6:10]]
        got = [int(w) for w in philox4x32_10(*ctr, *key)]
        assert got == out


def test_device_load_generator_equals_host():
    """loads_torch (the generator of the 10^9-DOF workload, run on the device
    there) draws the same Philox words and maps them the same way: bitwise the
    loads of `loads`, across chunk boundaries and 64-bit seeds."""
    torch = pytest.importorskip("torch")
    from workloads import loads_torch
    for nx, ny, seed, rhs, chunk in ((37, 29, 0, 0, 500), (64, 64, 5, 3, 1 << 20), (101, 7, 2**33 + 7, 1, 64)):
        assert np.array_equal(loads(nx, ny, seed, rhs), loads_torch(nx, ny, seed, rhs, chunk=chunk).numpy())


def test_load_and_ea_distributions():
    p = loads(300, 200, 5)
    assert p.shape == (200, 300, 2)
    assert p.min() > -1.0 and p.max() < 1.0
    assert abs(p.mean()) < 0.01 and abs(p.var() - 1.0 / 3.0) < 0.01
    ea = ea_lognormal(300, 200, 5)
    z = np.log(ea)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 0.3) < 0.01
    # counter-based: an entry does not depend on the lattice size
    assert np.array_equal(loads(10, 1, 5)[0], loads(10, 3, 5)[0])


# ---------------------------------------------------------------- stiffness
def brute_force_K(nx, ny, ea=None, L=1.0):
    """Dense K from node coordinates only: every pair of nodes at distance L
    is a rod; its owner is the lower node (or the left one in a row), its
    direction label E / NE / NW is read off the vector between them."""
    n = nx * ny
    xy = np.array([(L * (i + 0.5 * (j % 2)), L * j * SQ3 / 2) for j in range(ny) for i in range(nx)])
    K = np.zeros((2 * n, 2 * n))
    for a in range(n):
        for b in range(a + 1, n):
            d = xy[b] - xy[a]
            dist = math.hypot(*d)
            if abs(dist - L) > 1e-9:
                continue
            e = d / dist
            ja, ia = divmod(a, nx)
            if abs(d[1]) < 1e-12:
                lab = 0
            else:
                lab = 1 if d[0] > 0 else 2
            k = (1.0 if ea is None else ea[lab, ja, ia]) / L
            kee = k * np.outer(e, e)
            for (p, q, s) in ((a, a, 1), (b, b, 1), (a, b, -1), (b, a, -1)):
                K[2 * p:2 * p + 2, 2 * q:2 * q + 2] += s * kee
    return K


@pytest.mark.parametrize("nx,ny,lognormal", [(4, 3, False), (5, 4, True), (3, 6, True)])
def test_K_matches_brute_force(nx, ny, lognormal):
    ea = ea_lognormal(nx, ny, 3) if lognormal else None
    K = truss.assemble_K(nx, ny, ea).toarray()
    Kb = brute_force_K(nx, ny, ea)
    assert np.allclose(K, Kb, rtol=0, atol=1e-13)


def test_bar_count_and_coordination():
    nx, ny = 9, 8
    a, b, d = truss.bars(nx, ny)
    # every interior node has six neighbours
    deg = np.bincount(np.concatenate([a, b]), minlength=nx * ny).reshape(ny, nx)
    assert (deg[1:-1, 1:-1] == 6).all()
    # number of bars of a triangulated offset-row lattice
    assert len(a) == (nx - 1) * ny + (ny - 1) * (2 * nx - 1)


def test_K_symmetric_spd_and_rigid_modes():
    nx, ny = 7, 6
    tr = truss.Truss(nx, ny, ea_lognormal(nx, ny, 1))
    K = tr.K.toarray()
    assert np.allclose(K, K.T, atol=1e-14)
    w_free = np.linalg.eigvalsh(tr.K_ff().toarray())
    assert w_free.min() > 1e-6
    # unsupported: exactly the three rigid motions of the plane are free
    w = np.linalg.eigvalsh(K)
    assert (np.abs(w) < 1e-10).sum() == 3
    assert w[3] > 1e-4


def test_patch_test_affine_displacement():
    """A uniform strain field (affine u) gives zero force at every interior
    node for uniform EA; with non-uniform EA it does not."""
    nx, ny = 8, 7
    x, y = truss.node_xy(nx, ny)
    A = np.array([[0.3, -0.7], [0.2, 0.5]])
    c = np.array([1.5, -2.0])
    u = np.stack([A[0, 0] * x + A[0, 1] * y + c[0], A[1, 0] * x + A[1, 1] * y + c[1]], -1).reshape(-1)
    f = (truss.assemble_K(nx, ny) @ u).reshape(ny, nx, 2)
    assert np.abs(f[1:-1, 1:-1]).max() < 1e-12
    assert np.abs(f).max() > 1e-3  # boundary nodes are loaded
    f2 = (truss.assemble_K(nx, ny, ea_lognormal(nx, ny, 2)) @ u).reshape(ny, nx, 2)
    assert np.abs(f2[1:-1, 1:-1]).max() > 1e-3


def test_internal_forces_self_equilibrated():
    """Bar forces come in equal and opposite pairs along the bar: sum of
    forces and of moments of K u vanish for any u (unsupported K)."""
    nx, ny = 6, 5
    K = truss.assemble_K(nx, ny, ea_lognormal(nx, ny, 4))
    x, y = truss.node_xy(nx, ny)
    u = np.random.default_rng(0).standard_normal(2 * nx * ny)
    f = (K @ u).reshape(-1, 2)
    assert np.abs(f.sum(0)).max() < 1e-12
    mom = (x.reshape(-1) * f[:, 1] - y.reshape(-1) * f[:, 0]).sum()
    assert abs(mom) < 1e-11


# ---------------------------------------------------------------- O1 direct solve
@pytest.mark.parametrize("nx,ny,lognormal", [(9, 7, False), (12, 11, True)])
def test_direct_matches_dense_solve(nx, ny, lognormal):
    tr = truss.Truss(nx, ny, ea_lognormal(nx, ny, 9) if lognormal else None)
    p = tr.free * loads(nx, ny, 2).reshape(-1)
    u = direct.cholesky_solve(tr, p)
    Kf = tr.K_ff().toarray()
    uf = np.linalg.solve(Kf, p[tr.fdofs])
    assert np.allclose(u[tr.fdofs], uf, rtol=1e-12, atol=1e-12)
    assert np.all(u[~tr.free] == 0)


@pytest.mark.parametrize("nx,ny,lognormal", [(9, 7, False), (12, 11, True), (40, 33, True)])
def test_sparse_direct_matches_banded_and_dense(nx, ny, lognormal):
    """The sparse direct solve (used where the band no longer fits) against a
    dense solve and the banded Cholesky, and its residual against K itself."""
    tr = truss.Truss(nx, ny, ea_lognormal(nx, ny, 13) if lognormal else None)
    p = tr.free * loads(nx, ny, 4).reshape(-1)
    u = direct.sparse_solve(tr, p)
    assert np.all(u[~tr.free] == 0)
    ub = direct.cholesky_solve(tr, p)
    assert np.linalg.norm(u - ub) <= 1e-12 * np.linalg.norm(ub)
    if tr.fdofs.size <= 1000:
        uf = np.linalg.solve(tr.K_ff().toarray(), p[tr.fdofs])
        assert np.allclose(u[tr.fdofs], uf, rtol=1e-12, atol=1e-12)
    r = tr.residual(p, u)
    assert np.abs(r).sum() <= 1e-13 * np.abs(p).sum()


def test_reactions_balance_loads():
    """At the solution the supports carry the applied loads: K u summed over
    the constrained DOFs equals minus the sum of the loads (forces and moment)."""
    nx, ny = 10, 9
    tr = truss.Truss(nx, ny, ea_lognormal(nx, ny, 5))
    p = tr.free * loads(nx, ny, 3).reshape(-1)
    u = direct.cholesky_solve(tr, p)
    f = tr.reactions(u)
    assert np.abs((f - p)[tr.free]).max() < 1e-10
    fixed = (~tr.free).reshape(-1, 2)
    F = f.reshape(-1, 2) * fixed
    P = p.reshape(-1, 2)
    assert np.allclose(F.sum(0), -P.sum(0), atol=1e-9)
    x, y = tr.x.reshape(-1), tr.y.reshape(-1)
    mF = (x * F[:, 1] - y * F[:, 0]).sum()
    mP = (x * P[:, 1] - y * P[:, 0]).sum()
    assert mF == pytest.approx(-mP, abs=1e-8)


# ---------------------------------------------------------------- O2 iteration
def small_problem(nx=14, ny=12, sx=5, sy=4, lognormal=True, seed=0):
    tr = truss.Truss(nx, ny, ea_lognormal(nx, ny, seed + 11) if lognormal else None)
    g = hms.SetGrid(nx, ny, sx, sy)
    p = tr.free * loads(nx, ny, seed).reshape(-1)
    return tr, g, p


def test_relaxation_residual_form_equals_eq12():
    """delta_I = (k^Inner)^-1 r_I equals u^RD - u^old with u^RD from Eq. 12."""
    tr, g, p = small_problem()
    u = tr.free * np.random.default_rng(1).standard_normal(tr.ndof)
    lf = hms.LocalFactors(tr, g)
    delta = lf.relax(tr.residual(p, u))
    for I in (0, 4, g.M - 1):
        inner, urd = hms.relax_eq12(tr, g, p, u, I)
        assert np.allclose(delta[inner], urd - u[inner], rtol=1e-11, atol=1e-12)


def test_local_solve_residual():
    tr, g, p = small_problem()
    lf = hms.LocalFactors(tr, g)
    r = tr.residual(p, np.zeros(tr.ndof))
    delta = lf.relax(r)
    K = tr.K.tocsr()
    for d in lf.dofs:
        kin = K[d][:, d]
        assert np.allclose(kin @ delta[d], r[d], rtol=0, atol=1e-12 * np.abs(r).max())


def test_modes_by_construction():
    """Columns of V are the nine modes of Eqs. 9, 10, 13, 14 on the set's free DOFs."""
    tr, g, _ = small_problem(sx=5, sy=4)
    delta = tr.free * np.random.default_rng(2).standard_normal(tr.ndof)
    V = hms.modes(tr, g, delta).toarray()
    xc, yc = hms.rep_points(tr, g)
    ns = g.node_set().reshape(-1)
    for I in (0, 3, g.M - 1):
        for n in np.flatnonzero(ns == I):
            xi = tr.x.reshape(-1)[n] - xc[I]
            eta = tr.y.reshape(-1)[n] - yc[I]
            dx, dy = delta[2 * n], delta[2 * n + 1]
            want = [(1, 0), (0, 1), (xi, 0), (eta, 0), (0, xi), (0, eta), (dx, dy), (xi * dx, xi * dy),
                    (eta * dx, eta * dy)]
            for m, (wx, wy) in enumerate(want):
                gx = V[2 * n, 9 * I + m]
                gy = V[2 * n + 1, 9 * I + m]
                assert gx == pytest.approx(wx * tr.free[2 * n], abs=1e-14)
                assert gy == pytest.approx(wy * tr.free[2 * n + 1], abs=1e-14)
        # zero outside the set
        out = np.repeat(ns != I, 2)
        assert np.abs(V[out][:, 9 * I:9 * I + 9]).max() == 0


def test_coarse_system_dense_brute_force():
    """K_aa (Eq. 6) and P (Eq. 7) by dense triple sums over DOFs."""
    tr, g, p = small_problem(nx=9, ny=8, sx=4, sy=3)
    u = tr.free * np.random.default_rng(3).standard_normal(tr.ndof)
    r = tr.residual(p, u)
    delta = hms.LocalFactors(tr, g).relax(r)
    V = hms.modes(tr, g, delta).toarray()
    Kd = brute_force_K(tr.nx, tr.ny, tr.ea)
    Kd = Kd * np.outer(tr.free, tr.free)
    Kaa, P = hms.coarse_system(tr, hms.modes(tr, g, delta), r)
    Kb = np.einsum("im,ij,jl->ml", V, Kd, V)
    Pb = np.einsum("im,i->m", V, (tr.free * (p - Kd @ u)))
    assert np.allclose(Kaa, Kb, rtol=1e-12, atol=1e-10)
    assert np.allclose(P, Pb, rtol=1e-12, atol=1e-12)


def test_coarse_solve_special_cases():
    rng = np.random.default_rng(4)
    B = rng.standard_normal((12, 12))
    A = B @ B.T + 12 * np.eye(12)
    b = rng.standard_normal(12)
    a, dr = hms.coarse_solve(A, b)
    assert not dr.any()
    assert np.allclose(a, np.linalg.solve(A, b), rtol=1e-12)
    # an identically zero mode is dropped and the rest solve the reduced system
    A2 = A.copy()
    A2[5, :] = 0
    A2[:, 5] = 0
    a2, dr2 = hms.coarse_solve(A2, b)
    keep = np.arange(12) != 5
    assert dr2[5] and dr2.sum() == 1 and a2[5] == 0
    assert np.allclose(a2[keep], np.linalg.solve(A[np.ix_(keep, keep)], b[keep]), rtol=1e-12)
    # a mode that vanishes up to rounding (norm 1e-16 of its set's others) is dropped
    n9 = 18
    E = rng.standard_normal((n9, n9))
    E = E @ E.T + n9 * np.eye(n9)
    sc = np.ones(n9)
    sc[13] = 1e-16
    E = sc[:, None] * E * sc[None, :]
    be = sc * rng.standard_normal(n9)
    ae, dre = hms.coarse_solve(E, be)
    keep13 = np.arange(n9) != 13
    assert dre[13] and dre.sum() == 1 and ae[13] == 0
    assert np.allclose(ae[keep13], np.linalg.solve(E[np.ix_(keep13, keep13)], be[keep13]), rtol=1e-10)
    # a mode equal to twice another is dependent: the later one is dropped
    C = np.zeros((13, 13))
    C[:12, :12] = A
    C[12, :12] = 2 * A[3]
    C[:12, 12] = 2 * A[:, 3]
    C[12, 12] = 4 * A[3, 3]
    bb = np.append(b, 2 * b[3])
    a3, dr3 = hms.coarse_solve(C, bb)
    assert dr3[12] and dr3.sum() == 1
    assert np.allclose(a3[:12], np.linalg.solve(A, b), rtol=1e-10)


def test_one_set_is_a_direct_solve():
    """With the whole lattice as one set, delta = K^-1 r, so one update reaches
    u* with a_7 = 1 (Eqs. 12-13 over the whole domain)."""
    nx, ny = 11, 9
    tr = truss.Truss(nx, ny, ea_lognormal(nx, ny, 6))
    g = hms.SetGrid(nx, ny, nx, ny)
    p = tr.free * loads(nx, ny, 7).reshape(-1)
    res = hms.solve(tr, g, p, tol=1e-13, max_iter=1, keep_iterates=True)
    u_ref = direct.cholesky_solve(tr, p)
    assert np.linalg.norm(res.iterates[0] - u_ref) < 1e-10 * np.linalg.norm(u_ref)
    r = tr.residual(p, np.zeros(tr.ndof))
    delta = hms.LocalFactors(tr, g).relax(r)
    Kaa, P = hms.coarse_system(tr, hms.modes(tr, g, delta), r)
    a, _ = hms.coarse_solve(Kaa, P)
    assert a[6] == pytest.approx(1.0, abs=1e-9)


def test_energy_decreases_and_beats_plain_relaxation():
    """Pi of Eq. 2 decreases every iteration and never exceeds Pi(u + delta)."""
    tr, g, p = small_problem()
    lf = hms.LocalFactors(tr, g)
    res = hms.solve(tr, g, p, tol=1e-12, max_iter=25, keep_iterates=True, factors=lf)
    Pi = [h["Pi"] for h in res.history]
    assert all(b < a + 1e-12 * abs(a) for a, b in zip(Pi, Pi[1:]))
    u = np.zeros(tr.ndof)
    for un in res.iterates[:5]:
        plain = u + lf.relax(tr.residual(p, u))
        assert tr.energy(p, un) <= tr.energy(p, plain) + 1e-12 * abs(tr.energy(p, plain))
        u = un
    # the history's Pi is the energy of the iterate
    assert res.history[3]["Pi"] == pytest.approx(tr.energy(p, res.iterates[2]), rel=1e-12)


def test_galerkin_orthogonality():
    """After each update V^T r_new = 0 (Eq. 5 holds at the new iterate)."""
    tr, g, p = small_problem()
    lf = hms.LocalFactors(tr, g)
    u = np.zeros(tr.ndof)
    for _ in range(4):
        r = tr.residual(p, u)
        V = hms.modes(tr, g, lf.relax(r))
        Kaa, P = hms.coarse_system(tr, V, r)
        a, _ = hms.coarse_solve(Kaa, P)
        u = u + V @ a
        rn = tr.residual(p, u)
        assert np.abs(V.T @ rn).max() < 1e-9 * np.abs(V.T @ r).max()


def test_representing_node_invariance():
    """The modes' span does not depend on (x^(I), y^(I)) (Eq. 10), so neither do the iterates."""
    tr, g, p = small_problem()
    lf = hms.LocalFactors(tr, g)
    a = hms.solve(tr, g, p, tol=0, max_iter=6, keep_iterates=True, factors=lf)
    corner = (np.zeros(g.M) - 3.0, np.full(g.M, 7.5))
    b = hms.solve(tr, g, p, tol=0, max_iter=6, keep_iterates=True, rep=corner, factors=lf)
    for ua, ub in zip(a.iterates, b.iterates):
        assert np.linalg.norm(ua - ub) < 1e-9 * np.linalg.norm(ua)


def test_converges_to_direct_solution():
    nx, ny = 32, 32
    tr = truss.Truss(nx, ny)
    g = hms.SetGrid(nx, ny, 8, 8)
    p = tr.free * loads(nx, ny, 0).reshape(-1)
    res = hms.solve(tr, g, p, tol=1e-12, max_iter=500)
    assert res.converged
    u_ref = direct.cholesky_solve(tr, p)
    assert np.linalg.norm(res.u - u_ref) < 1e-9 * np.linalg.norm(u_ref)
    # the stop rule is Eq. 19's 1-norm relative residual
    r = tr.residual(p, res.u)
    assert np.abs(r).sum() / np.abs(p).sum() < 1e-12


def test_clamp_bottom_mask():
    f = clamp_bottom(5, 4)
    assert f[0].all() and not f[1:].any()
    assert np.array_equal(truss.free_mask(5, 4, f), truss.free_mask(5, 4, None))


# ---------------------------------------------------------------- planted mistakes
def test_pins_catch_a_wrong_bar_direction(monkeypatch):
    """Flipping the x component of the NE unit vector breaks the brute-force pin."""
    bad = truss.BAR_DIRS.copy()
    bad[1, 0] = -bad[1, 0]
    monkeypatch.setattr(truss, "BAR_DIRS", bad)
    K = truss.assemble_K(4, 3).toarray()
    assert not np.allclose(K, brute_force_K(4, 3), atol=1e-13)


def test_pins_catch_a_missing_gradient_factor(monkeypatch):
    """Dropping eta from mode 9 (eta*delta -> delta) duplicates mode 7; the
    dependent-mode rule then drops it and the energy pin still holds, but the
    mode-construction pin fails."""
    tr, g, _ = small_problem(sx=5, sy=4)
    orig = hms.modes

    def bad_modes(truss_, grid, delta, rep=None, mode_mask=0x1FF):
        V = orig(truss_, grid, delta, rep, mode_mask).tolil()
        for I in range(grid.M):
            V[:, 9 * I + 8] = V[:, 9 * I + 6]
        return V.tocsc()

    monkeypatch.setattr(hms, "modes", bad_modes)
    delta = tr.free * np.random.default_rng(2).standard_normal(tr.ndof)
    V = hms.modes(tr, g, delta).toarray()
    xc, yc = hms.rep_points(tr, g)
    n = np.flatnonzero(g.node_set().reshape(-1) == 0)[5]
    eta = tr.y.reshape(-1)[n] - yc[0]
    assert V[2 * n, 8] != pytest.approx(eta * delta[2 * n])


def test_pins_catch_a_sign_error_in_the_residual(monkeypatch):
    """r = p + K u instead of p - K u breaks convergence to the direct solution."""
    nx, ny = 12, 12
    tr = truss.Truss(nx, ny)
    g = hms.SetGrid(nx, ny, 4, 4)
    p = tr.free * loads(nx, ny, 0).reshape(-1)
    monkeypatch.setattr(truss.Truss, "residual", lambda self, p_, u_: self.free * (p_ + self.K @ (self.free * u_)))
    res = hms.solve(tr, g, p, tol=1e-10, max_iter=30)
    u_ref = direct.cholesky_solve(tr, p)
    assert not res.converged or np.linalg.norm(res.u - u_ref) > 1e-3 * np.linalg.norm(u_ref)


# ---------------------------------------------------------------- extended relaxation regions
def region_dofs(tr, g, I, e):
    """Free DOFs of set I's tile grown by e nodes, from node indices alone."""
    Ix, Iy = I % g.Mx, I // g.Mx
    i0, j0 = Ix * g.sx, Iy * g.sy
    out = []
    for n in range(tr.nx * tr.ny):
        i, j = n % tr.nx, n // tr.nx
        if i0 - e <= i < min(tr.nx, i0 + g.sx) + e and j0 - e <= j < min(tr.ny, j0 + g.sy) + e:
            out += [2 * n + c for c in range(2) if tr.free[2 * n + c]]
    return np.array(out)


@pytest.mark.parametrize("e", [1, 3])
def test_overlap_relaxation_solves_the_region(e):
    """delta_I is the solution of K restricted to the grown region (every other
    DOF held), taken on the set's own DOFs (Sec. 2.2, the extended region)."""
    tr = truss.Truss(13, 11, ea_lognormal(13, 11, 5))
    g = hms.SetGrid(13, 11, 5, 4)
    p = loads(13, 11, 9, 0).reshape(-1)
    r = tr.residual(p, np.zeros(tr.ndof))
    delta = hms.LocalFactors(tr, g, overlap=e).relax(r)
    K = tr.K.toarray()
    for I in (0, 4, g.M - 1):
        dr = region_dofs(tr, g, I, e)
        ds = region_dofs(tr, g, I, 0)
        sol = np.linalg.solve(K[np.ix_(dr, dr)], r[dr])
        want = sol[np.searchsorted(dr, ds)]
        assert np.allclose(delta[ds], want, rtol=0, atol=1e-11 * np.abs(want).max())


def test_overlap_covering_the_lattice_is_one_direct_update():
    """Grown over the whole lattice, every set's relaxation is the direct
    solution on its DOFs, so the modes delta_I add up to it and one update
    reaches it."""
    tr = truss.Truss(24, 20)
    g = hms.SetGrid(24, 20, 8, 8)
    p = loads(24, 20, 3, 0).reshape(-1)
    res = hms.solve(tr, g, p, 1e-12, 5, factors=hms.LocalFactors(tr, g, overlap=24))
    ref = direct.cholesky_solve(tr, tr.free * p)
    assert res.iterations == 1
    assert np.linalg.norm(res.u - ref) / np.linalg.norm(ref) < 1e-12


def test_overlap_reduces_iterations():
    """A larger relaxation region needs fewer updates (Sec. 2.2)."""
    tr = truss.Truss(24, 20)
    g = hms.SetGrid(24, 20, 8, 8)
    p = loads(24, 20, 3, 0).reshape(-1)
    nir = [hms.solve(tr, g, p, 1e-8, 500, factors=hms.LocalFactors(tr, g, overlap=e)).iterations
           for e in (0, 1, 4)]
    assert nir[0] > nir[1] > nir[2]


# ---------------------------------------------------------------- force-controlled relaxation
def brute_force_set_K(nx, ny, ea, members):
    """Dense stiffness of the rods with both ends in ``members`` (a set of node
    indices), from node coordinates only (as brute_force_K)."""
    n = nx * ny
    xy = np.array([(i + 0.5 * (j % 2), j * SQ3 / 2) for j in range(ny) for i in range(nx)])
    K = np.zeros((2 * n, 2 * n))
    for a in members:
        for b in members:
            if b <= a:
                continue
            d = xy[b] - xy[a]
            if abs(math.hypot(*d) - 1.0) > 1e-9:
                continue
            e = d
            ja, ia = divmod(a, nx)
            lab = 0 if abs(d[1]) < 1e-12 else (1 if d[0] > 0 else 2)
            kee = (1.0 if ea is None else ea[lab, ja, ia]) * np.outer(e, e)
            for (p, q, s) in ((a, a, 1), (b, b, 1), (a, b, -1), (b, a, -1)):
                K[2 * p:2 * p + 2, 2 * q:2 * q + 2] += s * kee
    return K


def force_problem():
    nx, ny = 18, 14
    ea = ea_lognormal(nx, ny, 21)
    return truss.Truss(nx, ny, ea), hms.SetGrid(nx, ny, 6, 5), ea


def test_force_matrix_is_the_stiffness_of_the_sets_own_bars():
    """k^Inner + Delta k (Eq. 15) = the set cut free: only the rods with both
    ends in the set act."""
    tr, g, ea = force_problem()
    ff = hms.ForceFactors(tr, g)
    ns = g.node_set().reshape(-1)
    for I in (0, 4, g.M - 1):
        members = [int(v) for v in np.flatnonzero(ns == I)]
        Kb = brute_force_set_K(tr.nx, tr.ny, ea, members)
        d = ff.dofs[I]
        assert np.allclose(ff.mats[I], Kb[np.ix_(d, d)], rtol=0, atol=1e-12)


def test_floating_set_null_space_is_the_rigid_motions():
    """A set clear of the supports has exactly the three rigid motions of the
    plane (two translations, the rotation) as zero modes; one on the clamped
    row has none."""
    tr, g, _ = force_problem()
    ff = hms.ForceFactors(tr, g)
    ns = g.node_set().reshape(-1)
    I = g.Mx + 1  # an interior set
    d = ff.dofs[I]
    assert d.size - ff.eig[I][0].size == 3
    nodes = d[0::2] // 2
    x, y = tr.x.reshape(-1)[nodes], tr.y.reshape(-1)[nodes]
    R = np.zeros((d.size, 3))
    R[0::2, 0] = 1.0
    R[1::2, 1] = 1.0
    R[0::2, 2], R[1::2, 2] = -y, x
    assert np.abs(ff.mats[I] @ R).max() < 1e-12
    assert ff.dofs[0].size == ff.eig[0][0].size  # the bottom-left set touches the clamp


def test_force_relaxation_is_the_minimum_norm_solution():
    """delta^RF_I solves the cut-free system for r_I with its rigid-motion part
    removed, and has no rigid-motion part itself (reading of the floating set)."""
    tr, g, _ = force_problem()
    ff = hms.ForceFactors(tr, g)
    r = tr.residual(loads(tr.nx, tr.ny, 4, 0).reshape(-1), np.zeros(tr.ndof))
    delta = ff.relax(r)
    I = g.Mx + 1
    d = ff.dofs[I]
    nodes = d[0::2] // 2
    x, y = tr.x.reshape(-1)[nodes], tr.y.reshape(-1)[nodes]
    R = np.zeros((d.size, 3))
    R[0::2, 0] = 1.0
    R[1::2, 1] = 1.0
    R[0::2, 2], R[1::2, 2] = -y, x
    Qr, _ = np.linalg.qr(R)
    rI = r[d] - Qr @ (Qr.T @ r[d])
    assert np.abs(Qr.T @ delta[d]).max() < 1e-10 * np.abs(delta[d]).max()
    assert np.allclose(ff.mats[I] @ delta[d], rI, rtol=0, atol=1e-10 * np.abs(rI).max())


def test_twelve_modes_converge_and_need_fewer_updates():
    """With the force-controlled modes (q = 12, Eqs. 17-18) the iteration still
    converges to the direct solution, keeps Galerkin orthogonality (Eq. 5) and
    needs fewer updates than with q = 9."""
    tr, g, _ = force_problem()
    p = loads(tr.nx, tr.ny, 7, 0).reshape(-1)
    ff = hms.ForceFactors(tr, g)
    r9 = hms.solve(tr, g, p, 1e-10, 2000)
    r12 = hms.solve(tr, g, p, 1e-10, 2000, force=ff, keep_iterates=True)
    ref = direct.cholesky_solve(tr, tr.free * p)
    assert r12.converged and np.linalg.norm(r12.u - ref) / np.linalg.norm(ref) < 1e-9
    assert r12.iterations < r9.iterations
    # Eq. 5 after the first update: V^T r_new = 0 for the twelve modes of that update
    r0 = tr.residual(tr.free * p, np.zeros(tr.ndof))
    V = hms.modes(tr, g, hms.LocalFactors(tr, g).relax(r0), delta_rf=ff.relax(r0))
    r1 = tr.residual(tr.free * p, r12.iterates[0])
    assert np.abs(V.T @ r1).max() < 1e-9 * np.abs(V.T @ r0).max()


def test_pool_relaxation_equals_serial():
    """The per-set relaxation spread over worker processes adds up to the serial
    one exactly (every DOF belongs to one set)."""
    from oracle import pool
    tr, g, p = small_problem(nx=23, ny=19, sx=6, sy=5)
    ea = ea_lognormal(23, 19, 11)
    r = tr.residual(p, np.zeros_like(p))
    ref = hms.LocalFactors(tr, g).relax(r)
    with pool.PoolFactors(23, 19, 6, 5, ea=ea, workers=3) as pf:
        got = pf.relax(r)
    assert np.array_equal(got, ref)
