"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Every step of one iteration (residual, update, relaxation, upper-level force,
matrix and solve) is compared element by element with the oracle on the same
seeded inputs, on lattices that span several set tiles with ragged edges, odd
row parity, one-row and one-column sets, a single set and a custom support
mask; then whole solves (trajectory and final displacement) and the error
paths.  Tolerances come from the arithmetic:

* FP64 steps: rounding-level, relative 1e-12 (a few ulps times the operation
  count); the local solves carry the local condition number (<= 1e4 here), so
  1e-11.
* Mixed path: the relaxation runs in FP32, so delta agrees to about
  kappa_local * 6e-8 (bound 2e-5); every later step is checked against the
  oracle fed the GPU's FP32-rounded delta, at FP64 level.
* Trajectories (T1): 1e-9 per iterate (FP64 path).
* Final displacement vs the direct solve (T2): 1e-9 (FP64), 1e-8 (mixed).
"""
import json
import os

import numpy as np
import pytest

from oracle import direct, hms, truss
from workloads import ea_lognormal, loads

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def left_and_bottom_fixed(nx, ny):
    f = np.zeros((ny, nx, 2), np.uint8)
    f[0] = 1
    f[:, 0, 0] = 1  # roller on the left edge: x only
    return f


# name, nx, ny, sx, sy, lognormal EA, fixed mask builder
CASES = [
    ("grid64_sets16", 64, 64, 16, 16, False, None),
    ("ragged_lognormal", 37, 29, 8, 6, True, None),
    ("odd_row_sets", 20, 13, 7, 5, False, None),
    ("widest_sets", 67, 24, 64, 12, True, None),
    ("roller_support", 24, 18, 6, 6, True, left_and_bottom_fixed),
    ("single_set", 12, 10, 12, 10, True, None),
    ("one_row_sets", 16, 9, 8, 1, False, None),
    ("one_column_sets", 9, 12, 1, 4, False, None),
]
PRECS = [0, 1]  # HMS_FP64, HMS_MIXED


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def setup_case(ctx, case, prec, tol=1e-11, max_iter=800, **kw):
    from paper_1208_4093_gb300 import capi
    name, nx, ny, sx, sy, ln, fixb = case
    ea = ea_lognormal(nx, ny, 17) if ln else None
    fixed = fixb(nx, ny) if fixb else None
    tr = truss.Truss(nx, ny, ea, fixed)
    g = hms.SetGrid(nx, ny, sx, sy)
    p = loads(nx, ny, 5).reshape(-1)
    pr = capi.hms_problem_create(ctx, nx, ny, sx, sy, ea=ea, fixed=fixed, precision=prec, tol=tol,
                                 max_iter=max_iter, **kw)
    return tr, g, p, pr


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


@pytest.fixture(params=[(c, p) for c in CASES for p in PRECS], ids=lambda cp: f"{cp[0][0]}-{'mixed' if cp[1] else 'fp64'}")
def problem(request, hms_ctx):
    from paper_1208_4093_gb300 import capi
    case, prec = request.param
    tr, g, p, pr = setup_case(hms_ctx, case, prec)
    yield hms_ctx, case, prec, tr, g, p, pr
    capi.hms_problem_destroy(pr)


def test_residual_step(problem):
    from paper_1208_4093_gb300 import capi
    ctx, case, prec, tr, g, p, pr = problem
    u = np.random.default_rng(1).standard_normal(tr.ndof)  # nonzero on constrained DOFs too
    r = np.empty(tr.ndof)
    nrm = np.empty(3)
    capi.hms_residual(ctx, pr, p, u, r, nrm)
    uf = tr.free * u
    ro = tr.residual(tr.free * p, uf)
    assert rel(r, ro) < 1e-13
    assert np.all(r[~tr.free] == 0)
    assert nrm[0] == pytest.approx(np.abs(ro).sum(), rel=1e-13)
    assert nrm[1] == pytest.approx(ro @ ro, rel=1e-13)
    assert nrm[2] == pytest.approx(uf @ (tr.free * p + ro), rel=1e-12)


def test_update_residual_step(problem):
    from paper_1208_4093_gb300 import capi
    ctx, case, prec, tr, g, p, pr = problem
    rng = np.random.default_rng(2)
    u = tr.free * rng.standard_normal(tr.ndof)
    delta = tr.free * rng.standard_normal(tr.ndof)
    a = rng.standard_normal(9 * g.M)
    uo, r, nrm = np.empty(tr.ndof), np.empty(tr.ndof), np.empty(3)
    capi.hms_update_residual(ctx, pr, p, u, delta, a, uo, r, nrm)
    d_used = f32(delta) if prec == 1 else delta  # the mixed path stores delta in FP32
    V = hms.modes(tr, g, d_used)
    un = u + V @ a
    if prec == 0:
        assert rel(uo, un) < 1e-13
    else:
        # the mixed form adds an FP32 increment: a few FP32 roundings of terms
        # bounded by sum_m |a_m| |mode_m| at each DOF (2^-24 ~ 6e-8 each)
        bound = 1e-6 * (abs(V) @ np.abs(a))
        assert np.all(np.abs(uo - un) <= bound + 1e-300)
        assert rel(uo, un) < 1e-6
    # r is the residual of the u the kernel wrote
    assert rel(r, tr.residual(tr.free * p, uo)) < 1e-12


def test_relax_step(problem):
    from paper_1208_4093_gb300 import capi
    ctx, case, prec, tr, g, p, pr = problem
    u = tr.free * np.random.default_rng(3).standard_normal(tr.ndof)
    r = tr.residual(tr.free * p, u)
    dl, P = np.empty(tr.ndof), np.empty(9 * g.M)
    capi.hms_relax(ctx, pr, r, dl, P)
    do = hms.LocalFactors(tr, g).relax(r)
    assert rel(dl, do) < (2e-5 if prec == 1 else 1e-11)
    assert np.all(dl[~tr.free] == 0)
    # P = V^T r (Eq. 7) with the modes of the delta the GPU produced
    Po = hms.modes(tr, g, dl).T @ r
    assert rel(P, Po) < 1e-12


def test_coarse_matrix_step(problem):
    from paper_1208_4093_gb300 import capi
    ctx, case, prec, tr, g, p, pr = problem
    if 9 * g.M > 4096:
        pytest.skip("dense K_aa only for small set grids")
    u = tr.free * np.random.default_rng(4).standard_normal(tr.ndof)
    r = tr.residual(tr.free * p, u)
    delta = hms.LocalFactors(tr, g).relax(r)
    Kaa = np.empty((9 * g.M, 9 * g.M))
    capi.hms_coarse_matrix(ctx, pr, delta, Kaa)
    d_used = f32(delta) if prec == 1 else delta
    Ko, _ = hms.coarse_system(tr, hms.modes(tr, g, d_used), r)
    # FP64 path: rounding level.  Mixed path: the delta-mode products of bars
    # inside a set run in FP32 (FP64 sums across threads), ~1e-7 per product
    assert np.abs(Kaa - Ko).max() < (1e-5 if prec == 1 else 1e-12) * np.abs(Ko).max()
    assert np.array_equal(Kaa, Kaa.T)


def test_coarse_solve_step(problem):
    from paper_1208_4093_gb300 import capi
    ctx, case, prec, tr, g, p, pr = problem
    if 9 * g.M > 4096:
        pytest.skip("dense K_aa only for small set grids")
    u = tr.free * np.random.default_rng(5).standard_normal(tr.ndof)
    r = tr.residual(tr.free * p, u)
    # zero residual on set 0: its relaxation modes vanish and must be dropped
    ns = np.repeat(g.node_set().reshape(-1), 2)
    r[ns == 0] = 0.0
    delta = hms.LocalFactors(tr, g).relax(r)
    V = hms.modes(tr, g, delta)
    Ko, Po = hms.coarse_system(tr, V, r)
    a, dr = np.empty(9 * g.M), np.zeros(9 * g.M, np.int32)
    capi.hms_coarse_solve(ctx, pr, Ko, Po, a, dr)
    ao, dro = hms.coarse_solve(Ko, Po)
    dr = dr.astype(bool)
    zero_diag = ~(np.diag(Ko) > 1e-300)
    # modes that vanish identically are dropped by both
    assert np.array_equal(dr & zero_diag, zero_diag) and np.array_equal(dro & zero_diag, zero_diag)
    # the update V a (the energy minimiser over the modes' span) is unique
    # FP32 factor + FP64 refinement: 3 solves (FP64 path) reach ~1e-13, 2 solves
    # (mixed path) ~(kappa eps32)^2 <= 1e-6
    tol = 1e-11 if prec == 0 else 1e-6
    assert rel(V @ a, V @ ao) < max(tol, 1e-9)
    # Galerkin condition (Eq. 5) on the modes the GPU kept
    gal = (Po - Ko @ a)[~dr]
    assert np.abs(gal).max() <= max(tol, 1e-9) * np.abs(Po).max()
    # exactly dependent modes are decided by FP64 pivots at rounding level on
    # both sides; which one of a dependent group is dropped can differ where a
    # pivot sits at the threshold, and then only V a is unique (checked above)
    if not ((dro | dr) & ~zero_diag).any():
        assert np.array_equal(dr, dro)
        assert rel(a, ao) < tol


@pytest.mark.parametrize("cf", [1, 3, 4], ids=["cluster", "rows16", "onesm_blocks64"])
@pytest.mark.parametrize("case", [CASES[0], CASES[1], CASES[3]], ids=lambda c: c[0])
def test_coarse_solve_both_substitutions(hms_ctx, case, cf):
    """The FP32 factor on a cluster of SMs or on one SM, and its two
    substitutions (inverted 64 x 64 diagonal blocks, or 16-row steps), give the
    oracle's update V a and full solve."""
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup_case(hms_ctx, case, 0, coarse_factor=cf)
    try:
        u = tr.free * np.random.default_rng(9).standard_normal(tr.ndof)
        r = tr.residual(tr.free * p, u)
        delta = hms.LocalFactors(tr, g).relax(r)
        V = hms.modes(tr, g, delta)
        Ko, Po = hms.coarse_system(tr, V, r)
        a = np.empty(9 * g.M)
        capi.hms_coarse_solve(hms_ctx, pr, Ko, Po, a)
        ao, _ = hms.coarse_solve(Ko, Po)
        assert rel(V @ a, V @ ao) < 1e-11
        out = np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), out)
        assert rel(out[0], direct.cholesky_solve(tr, tr.free * p)) < 1e-9
    finally:
        capi.hms_problem_destroy(pr)


# set grids whose upper-level system is long enough to split: separator s =
# bw + 1 (33 x 90), bw + 4 (50 x 70), and a longer one (64 x 128)
TWO_SIDED = [
    ("split_s_bw1", 33, 90, 7, 6, True, None),
    ("split_s_bw4", 50, 70, 10, 7, False, None),
    ("split_long", 64, 128, 8, 8, True, None),
]


@pytest.mark.parametrize("case", TWO_SIDED + [CASES[1]], ids=lambda c: c[0])
def test_two_sided_factor(hms_ctx, case):
    """The FP32 factor of Eq. 8 split into top and bottom segments eliminated
    on two SMs and the separator between them: the update V a and the full
    solve match the oracle, and the result equals the one-SM factor's within
    the FP64 refinement's accuracy."""
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup_case(hms_ctx, case, 0, coarse_factor=5)
    pr1 = setup_case(hms_ctx, case, 0, coarse_factor=4)[3]
    try:
        rng = np.random.default_rng(19)
        for _ in range(2):
            u = tr.free * rng.standard_normal(tr.ndof)
            r = tr.residual(tr.free * p, u)
            delta = hms.LocalFactors(tr, g).relax(r)
            V = hms.modes(tr, g, delta)
            Ko, Po = hms.coarse_system(tr, V, r)
            a = np.empty(9 * g.M)
            a1 = np.empty(9 * g.M)
            dr = np.zeros(9 * g.M, np.int32)
            capi.hms_coarse_solve(hms_ctx, pr, Ko, Po, a, dropped_out=dr)
            capi.hms_coarse_solve(hms_ctx, pr1, Ko, Po, a1)
            ao, dro = hms.coarse_solve(Ko, Po)
            assert rel(V @ a, V @ ao) < 1e-11
            assert rel(V @ a, V @ a1) < 1e-11
            assert np.array_equal(dr != 0, np.asarray(dro, bool))
        out = np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), out)
        assert rel(out[0], direct.cholesky_solve(tr, tr.free * p)) < 1e-9
    finally:
        capi.hms_problem_destroy(pr)
        capi.hms_problem_destroy(pr1)


def test_two_sided_short_segment_block_converges(hms_ctx):
    """8 x 8 sets of 16 x 16 nodes: the bottom segment has 244 pivots, so its
    last 16-column block is short and rows of the separator follow it.  The
    panel of that block must not read the window positions right of those
    rows' band (never loaded: whatever an earlier kernel left in shared
    memory), which once turned this solve non-finite after ~105 updates."""
    from paper_1208_4093_gb300 import capi
    nx = 128
    tr = truss.Truss(nx, nx)
    p = loads(nx, nx, 0).reshape(-1)
    pr = capi.hms_problem_create(hms_ctx, nx, nx, 16, 16, precision=capi.HMS_FP64, tol=1e-10, max_iter=5000,
                                 coarse_factor=5)
    try:
        u = np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u)
        assert rel(u[0], direct.cholesky_solve(tr, tr.free * p)) < 1e-9
    finally:
        capi.hms_problem_destroy(pr)


def test_two_sided_needs_a_long_system(hms_ctx):
    """coarse_factor = 5 is refused where the system is shorter than two 64-row
    segments plus a separator (4 x 4 sets: n = 144, bw = 53)."""
    from paper_1208_4093_gb300 import capi
    with pytest.raises(capi.HmsError) as e:
        setup_case(hms_ctx, CASES[0], 0, coarse_factor=5)
    assert e.value.status == capi.HMS_ERR_ARG


def test_one_iteration_from_any_state(problem):
    """T1 per step: one GPU update from u equals one oracle update from u."""
    from paper_1208_4093_gb300 import capi
    ctx, case, prec, tr, g, p, pr = problem
    if prec == 1:
        pytest.skip("mixed-path steps differ from the FP64 oracle by design (FP32 delta)")
    lf = hms.LocalFactors(tr, g)
    u = np.zeros(tr.ndof)
    pr1 = setup_case(ctx, case, prec, tol=0.0, max_iter=1)[3]
    try:
        for _ in range(3):
            out = np.empty((1, tr.ndof))
            capi.hms_solve(ctx, pr1, p.reshape(1, -1), out, u0=u.reshape(1, -1), allow_no_convergence=True)
            want = hms.solve(tr, g, p, tol=0.0, max_iter=1, u0=u, factors=lf).u
            assert rel(out[0], want) < 1e-9
            u = want
    finally:
        capi.hms_problem_destroy(pr1)


def test_full_solve_matches_direct(problem):
    """T2: the converged displacement equals the direct solve; FP64 iteration
    counts equal the oracle's."""
    from paper_1208_4093_gb300 import capi
    ctx, case, prec, tr, g, p, pr = problem
    u = np.empty((1, tr.ndof))
    hist = np.full((1, 801, 3), np.nan)
    its = np.zeros(1, np.int32)
    capi.hms_solve(ctx, pr, p.reshape(1, -1), u, hist=hist, iters=its)
    u_ref = direct.cholesky_solve(tr, tr.free * p)
    assert rel(u[0], u_ref) < (1e-8 if prec == 1 else 1e-9)
    assert hist[0, its[0], 0] < 1e-11
    if prec == 0:
        res = hms.solve(tr, g, p, 1e-11, 800)
        assert abs(int(its[0]) - res.iterations) <= 1
        n = min(int(its[0]), res.iterations)
        ho = np.array([[h["R1"], h["R2"], h["Pi"]] for h in res.history[:n + 1]])
        hg = hist[0, :n + 1]
        # residual norms agree to rounding while they are well above the
        # rounding floor (~1e-16 |K u| / |p|); the energy agrees throughout
        big = ho[:, 0] > 1e-8
        assert np.allclose(hg[big, :2], ho[big, :2], rtol=1e-6)
        assert np.allclose(hg[:, 2], ho[:, 2], rtol=1e-10)


def test_lattice64_history_golden(hms_ctx):
    """The 64 x 64 lattice, 4 x 4 sets, tol 1e-8: iteration counts and residual
    histories of four load cases against the stored oracle run."""
    from paper_1208_4093_gb300 import capi
    d = json.load(open(os.path.join(GOLDEN, "lattice64_history.json")))
    pr = capi.hms_problem_create(hms_ctx, d["nx"], d["ny"], d["sx"], d["sy"], tol=d["tol"], max_iter=1000)
    try:
        for seed, rec in d["seeds"].items():
            p = loads(d["nx"], d["ny"], int(seed)).reshape(1, -1)
            u = np.empty_like(p)
            hist = np.full((1, 1001, 3), np.nan)
            its = np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr, p, u, hist=hist, iters=its)
            assert int(its[0]) == rec["iterations"]
            h = np.array(rec["history"])
            assert np.allclose(hist[0, :40], h[:40], rtol=1e-9)
            assert np.allclose(hist[0, :len(h), 0], h[:, 0], rtol=1e-4)
    finally:
        capi.hms_problem_destroy(pr)


# ---------------------------------------------------------------- solver behaviour
def test_multiple_rhs_and_determinism(hms_ctx):
    from paper_1208_4093_gb300 import capi
    case = CASES[1]
    tr, g, p, pr = setup_case(hms_ctx, case, 0, tol=1e-10)
    try:
        P = np.stack([loads(tr.nx, tr.ny, s).reshape(-1) for s in (1, 2)])
        U = np.empty_like(P)
        its = np.zeros(2, np.int32)
        capi.hms_solve(hms_ctx, pr, P, U, iters=its)
        for k in range(2):
            u1 = np.empty((1, tr.ndof))
            capi.hms_solve(hms_ctx, pr, P[k:k + 1], u1)
            assert np.array_equal(u1[0], U[k])  # bitwise: fixed-order reductions
    finally:
        capi.hms_problem_destroy(pr)


def test_device_pointers_match_host(hms_ctx):
    import torch
    from paper_1208_4093_gb300 import capi
    case = CASES[0]
    for prec in PRECS:
        tr, g, p, pr = setup_case(hms_ctx, case, prec, tol=1e-9)
        try:
            uh = np.empty((1, tr.ndof))
            capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), uh)
            pd = torch.from_numpy(p.reshape(1, -1)).cuda()
            ud = torch.empty_like(pd)
            capi.hms_solve(hms_ctx, pr, pd, ud)
            torch.cuda.synchronize()
            assert np.array_equal(ud.cpu().numpy(), uh)
        finally:
            capi.hms_problem_destroy(pr)


def test_max_iter_returns_last_iterate(hms_ctx):
    from paper_1208_4093_gb300 import capi
    case = CASES[2]
    tr, g, p, pr = setup_case(hms_ctx, case, 0, tol=1e-14, max_iter=7)
    try:
        u = np.empty((1, tr.ndof))
        its = np.zeros(1, np.int32)
        with pytest.raises(capi.HmsError) as ei:
            capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u, iters=its)
        assert ei.value.status == capi.HMS_ERR_NO_CONVERGENCE
        st = capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u, iters=its, allow_no_convergence=True)
        assert st == capi.HMS_ERR_NO_CONVERGENCE and its[0] == 7
        want = hms.solve(tr, g, p, 1e-14, 7).u
        assert rel(u[0], want) < 1e-9
    finally:
        capi.hms_problem_destroy(pr)


def test_zero_load_converges_immediately(hms_ctx):
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup_case(hms_ctx, CASES[2], 0)
    try:
        u = np.full((1, tr.ndof), 7.0)
        its = np.zeros(1, np.int32)
        capi.hms_solve(hms_ctx, pr, np.zeros((1, tr.ndof)), u, iters=its)
        assert its[0] == 0 and np.all(u == 0)
    finally:
        capi.hms_problem_destroy(pr)


def test_nonfinite_load_is_reported(hms_ctx):
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup_case(hms_ctx, CASES[2], 0)
    try:
        q = p.copy()
        q[-7] = np.nan  # a free DOF of the top row
        u = np.empty((1, tr.ndof))
        with pytest.raises(capi.HmsError) as ei:
            capi.hms_solve(hms_ctx, pr, q.reshape(1, -1), u)
        assert ei.value.status == capi.HMS_ERR_NONFINITE
    finally:
        capi.hms_problem_destroy(pr)


def test_singular_local_matrix_is_reported(hms_ctx):
    """One set covering an unsupported lattice: k^Inner = K is singular."""
    from paper_1208_4093_gb300 import capi
    with pytest.raises(capi.HmsError) as ei:
        capi.hms_problem_create(hms_ctx, 6, 5, 6, 5, fix_bottom_edge=0)
    assert ei.value.status == capi.HMS_ERR_NOT_SPD


@pytest.mark.parametrize("kw", [dict(nx=1), dict(sx=65), dict(sy=0), dict(ea_bad=True), dict(prec=7)])
def test_bad_arguments_rejected(hms_ctx, kw):
    from paper_1208_4093_gb300 import capi
    nx = kw.get("nx", 8)
    ea = None
    if kw.get("ea_bad"):
        ea = np.ones((3, 8, nx))
        ea[0, 2, 3] = -1.0
    with pytest.raises(capi.HmsError) as ei:
        capi.hms_problem_create(hms_ctx, nx, 8, kw.get("sx", 4), kw.get("sy", 4), ea=ea,
                                precision=kw.get("prec", 0))
    assert ei.value.status == capi.HMS_ERR_ARG


def test_wide_set_grid_needs_the_cluster_factor(hms_ctx):
    """24 sets across give bw = 9 * 26 - 1 = 233: one SM's window cannot hold
    the band, the factor on a cluster of SMs can, and the solve matches the
    direct solution."""
    from paper_1208_4093_gb300 import capi
    nx, ny, sx, sy = 96, 8, 4, 4
    with pytest.raises(capi.HmsError) as e:
        capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, coarse_factor=4)
    assert e.value.status == capi.HMS_ERR_ARG
    tr = truss.Truss(nx, ny)
    p = loads(nx, ny, 21).reshape(-1)
    pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, precision=capi.HMS_FP64, tol=1e-11, max_iter=20000)
    try:
        u = np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u)
        assert rel(u[0], direct.cholesky_solve(tr, tr.free * p)) < 1e-9
    finally:
        capi.hms_problem_destroy(pr)
