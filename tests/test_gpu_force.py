"""The force-controlled relaxation and the q = 12 modes of Eqs. 15-18 on the
GPU, against the oracle (``oracle.hms.ForceFactors``: the set cut free,
floating sets by the minimum-norm reading; ``solve(..., force=...)``).

mode_mask bits 9-11 turn the modes 10-12 on.  Tolerances: the force-
controlled solve of a floating set is the minimum-norm solution of a
singular system (GPU: pinned DOFs and a projection; oracle: an
eigendecomposition), so it agrees to the cut-free matrix's conditioning
(1e-8 FP64); every later step is checked at FP64 level on the GPU's own
deltas; whole solves against the direct solve (1e-9 FP64, 1e-8 mixed).
"""
import numpy as np
import pytest

from oracle import direct, hms, truss
from workloads import ea_lognormal, loads

pytestmark = pytest.mark.gpu

FORCE = 0xFFF


def left_and_bottom_fixed(nx, ny):
    f = np.zeros((ny, nx, 2), np.uint8)
    f[0] = 1
    f[:, 0, 0] = 1
    return f


# name, nx, ny, sx, sy, lognormal EA, fixed mask builder
CASES = [
    ("grid48_sets16", 48, 48, 16, 16, False, None),
    ("ragged_lognormal", 37, 29, 8, 6, True, None),
    ("odd_rows", 26, 22, 7, 5, False, None),
    ("roller_support", 24, 18, 6, 6, True, left_and_bottom_fixed),
    ("two_wide_sets", 20, 16, 2, 4, True, None),
]


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def setup(ctx, case, prec, **kw):
    from paper_1208_4093_gb300 import capi
    name, nx, ny, sx, sy, ln, fixb = case
    ea = ea_lognormal(nx, ny, 41) if ln else None
    fixed = fixb(nx, ny) if fixb else None
    tr = truss.Truss(nx, ny, ea, fixed)
    g = hms.SetGrid(nx, ny, sx, sy)
    p = tr.free * loads(nx, ny, 7).reshape(-1)
    pr = capi.hms_problem_create(ctx, nx, ny, sx, sy, ea=ea, fixed=fixed, precision=prec, mode_mask=FORCE, **kw)
    return tr, g, p, pr


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("prec", [0, 1])
def test_force_relaxation_matches_oracle(hms_ctx, case, prec):
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup(hms_ctx, case, prec)
    try:
        u = tr.free * np.random.default_rng(5).standard_normal(tr.ndof)
        r = tr.residual(p, u)
        d = np.empty_like(r)
        capi.hms_relax_force(hms_ctx, pr, r, d)
    finally:
        capi.hms_problem_destroy(pr)
    ref = hms.ForceFactors(tr, g).relax(r)
    assert np.all(d[~tr.free] == 0)
    assert rel(d, ref) < (1e-8 if prec == 0 else 1e-3), case[0]


@pytest.mark.parametrize("case", CASES[:4], ids=lambda c: c[0])
def test_relax_P_and_coarse_matrix_q12(hms_ctx, case):
    """P = V^T r and K_aa = V^T K V with the twelve modes, from the GPU's own
    deltas, against the oracle's sparse products (FP64 path)."""
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup(hms_ctx, case, 0)
    try:
        u = tr.free * np.random.default_rng(6).standard_normal(tr.ndof)
        r = tr.residual(p, u)
        d, drf = np.empty_like(r), np.empty_like(r)
        P = np.empty(12 * g.M)
        capi.hms_relax(hms_ctx, pr, r, d, P)
        capi.hms_relax_force(hms_ctx, pr, r, drf)
        V = hms.modes(tr, g, d, delta_rf=drf)
        Ko, Po = hms.coarse_system(tr, V, r)
        assert rel(P, Po) < 1e-12
        K = np.empty((12 * g.M, 12 * g.M))
        capi.hms_coarse_matrix(hms_ctx, pr, np.concatenate([d, drf]), K)
        assert np.abs(K - Ko).max() <= 1e-12 * np.abs(Ko).max()
        # the update u + V a with both increments
        a = np.random.default_rng(7).standard_normal(12 * g.M)
        uo, ro, nrm = np.empty_like(r), np.empty_like(r), np.empty(3)
        capi.hms_update_residual(hms_ctx, pr, p, u, np.concatenate([d, drf]), a, uo, ro, nrm)
        un = u + V @ a
        assert rel(uo, un) < 1e-13
        assert rel(ro, tr.residual(p, un)) < 1e-12
    finally:
        capi.hms_problem_destroy(pr)


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("prec", [0, 1])
def test_q12_solve_reaches_direct_solution(hms_ctx, case, prec):
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup(hms_ctx, case, prec, tol=1e-11, max_iter=3000)
    try:
        out = np.empty((1, tr.ndof))
        its = np.zeros(1, np.int32)
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), out, iters=its)
    finally:
        capi.hms_problem_destroy(pr)
    assert rel(out[0], direct.cholesky_solve(tr, p)) < (1e-9 if prec == 0 else 1e-8), case[0]


@pytest.mark.parametrize("case", CASES[:3], ids=lambda c: c[0])
def test_q12_trajectory_and_fewer_updates(hms_ctx, case):
    """The FP64 iterates follow the oracle's q = 12 iteration, and q = 12 needs
    fewer updates than q = 9 to the same tolerance (as in the oracle)."""
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = setup(hms_ctx, case, 0, tol=0.0, max_iter=3)
    ff = hms.ForceFactors(tr, g)
    try:
        out = np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), out, allow_no_convergence=True)
    finally:
        capi.hms_problem_destroy(pr)
    ref = hms.solve(tr, g, p, 0.0, 3, force=ff).u
    assert rel(out[0], ref) < 1e-7, case[0]
    its = {}
    for mask in (0x1FF, FORCE):
        name, nx, ny, sx, sy, ln, fixb = case
        pr2 = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, ea=ea_lognormal(nx, ny, 41) if ln else None,
                                      fixed=fixb(nx, ny) if fixb else None, tol=1e-8, max_iter=3000, mode_mask=mask)
        try:
            n = np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr2, p.reshape(1, -1), np.empty((1, tr.ndof)), iters=n)
            its[mask] = int(n[0])
        finally:
            capi.hms_problem_destroy(pr2)
    nor = hms.solve(tr, g, p, 1e-8, 3000, force=ff).iterations
    assert its[FORCE] < its[0x1FF]
    assert abs(its[FORCE] - nor) <= max(2, nor // 20)


def test_force_modes_need_two_by_two_sets(hms_ctx):
    from paper_1208_4093_gb300 import capi
    for args, kw in (((16, 9, 8, 1), {}), ((9, 12, 1, 4), {}), ((17, 12, 8, 4), {}),
                     ((40, 40, 16, 16), {"relax_overlap": 2, "precision": 1})):
        with pytest.raises(capi.HmsError) as e:
            capi.hms_problem_create(hms_ctx, *args, mode_mask=FORCE, **kw)
        assert e.value.status == capi.HMS_ERR_ARG


@pytest.mark.parametrize("prec", [0, 1])
def test_q12_on_a_wide_set_grid(hms_ctx, prec):
    """Twelve modes per set on a grid 40 sets across (no band factor fits:
    nested dissection of the set grid), against the direct solve."""
    from paper_1208_4093_gb300 import capi
    nx, ny = 320, 40
    ea = ea_lognormal(nx, ny, 43)
    tr = truss.Truss(nx, ny, ea)
    p = tr.free * loads(nx, ny, 9).reshape(-1)
    pr = capi.hms_problem_create(hms_ctx, nx, ny, 8, 10, ea=ea, precision=prec, mode_mask=FORCE, tol=1e-11,
                                 max_iter=4000)
    try:
        out = np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), out)
    finally:
        capi.hms_problem_destroy(pr)
    assert rel(out[0], direct.sparse_solve(tr, p)) < (1e-9 if prec == 0 else 1e-8)
