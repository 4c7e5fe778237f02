"""The relaxation with class factors (one factor per class of identical sets,
many sets' right-hand sides per CTA) against the oracle.

With a uniform bar stiffness, sets of the same shape, first-row parity,
lattice edges touched and supports share k^Inner (Eq. 12), so their local
solves are one matrix applied to many right-hand sides.  The oracle factors
every set on its own (LocalFactors), so agreement also shows that the sets
the library puts in one class really have the same matrix.  Tolerances as in
test_gpu_parity: FP64 1e-11 (local solves carry kappa_local), FP32 2e-5;
whole solves against the direct solve at 1e-9 (FP64) and 1e-8 (mixed).
"""
import numpy as np
import pytest

from oracle import direct, hms, truss
from workloads import loads

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def roller_left(nx, ny):
    f = np.zeros((ny, nx, 2), np.uint8)
    f[0] = 1
    f[:, 0, 0] = 1
    return f


def pinned_spots(nx, ny):
    # supports scattered inside the lattice: sets differ by their supports
    f = np.zeros((ny, nx, 2), np.uint8)
    f[0] = 1
    f[ny // 2, nx // 3] = 1
    f[ny - 1, nx - 1, 1] = 1
    return f


# name, nx, ny, sx, sy, fixed mask builder
CASES = [
    ("grid64_sets16", 64, 64, 16, 16, None),              # 3 x 3 edge classes, 16 sets
    ("ragged_both", 71, 45, 16, 12, None),                # ragged last column and row
    ("odd_set_rows", 40, 33, 8, 5, None),                 # odd sy: first-row parity alternates
    ("many_sets", 98, 90, 4, 4, None),                    # 25 x 23 sets: classes of several CTAs
    ("widest_sets", 140, 20, 64, 7, None),                # 64-node sets (nb = 128), ragged 12
    ("roller", 30, 26, 6, 6, roller_left),
    ("scattered_supports", 48, 40, 8, 8, pinned_spots),   # supports split classes
    ("one_node_wide", 9, 12, 1, 4, None),
    # the set shapes of the 22361 x 22361 lattice: 64 x 64-node sets, the
    # last row and column of sets 25 nodes wide, bottom row clamped
    ("paper_scale_shapes", 217, 217, 64, 64, None),
]
PRECS = [0, 1]


def make(ctx, case, prec, **kw):
    from paper_1208_4093_gb300 import capi
    name, nx, ny, sx, sy, fixb = case
    fixed = fixb(nx, ny) if fixb else None
    tr = truss.Truss(nx, ny, None, fixed)
    g = hms.SetGrid(nx, ny, sx, sy)
    pr = capi.hms_problem_create(ctx, nx, ny, sx, sy, fixed=fixed, precision=prec, class_factors=1, **kw)
    return tr, g, pr


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
def test_class_relax_step(hms_ctx, case, prec):
    """delta = (k^Inner)^-1 r for every set (Eq. 13) and P = V^T r (Eq. 7)."""
    from paper_1208_4093_gb300 import capi
    tr, g, pr = make(hms_ctx, case, prec, tol=1e-10, max_iter=10)
    try:
        for seed in (3, 4):
            u = tr.free * np.random.default_rng(seed).standard_normal(tr.ndof)
            p = loads(tr.nx, tr.ny, seed).reshape(-1)
            r = tr.residual(tr.free * p, u)
            dl, P = np.empty(tr.ndof), np.empty(9 * g.M)
            capi.hms_relax(hms_ctx, pr, r, dl, P)
            do = hms.LocalFactors(tr, g).relax(r)
            assert rel(dl, do) < (2e-5 if prec == 1 else 1e-11)
            assert np.all(dl[~tr.free] == 0)
            Po = hms.modes(tr, g, dl).T @ r
            assert rel(P, Po) < 1e-12
    finally:
        capi.hms_problem_destroy(pr)


@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[5], CASES[6], CASES[8]], ids=lambda c: c[0])
@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
def test_class_solve_matches_direct(hms_ctx, case, prec):
    """Whole solves to R1 < 1e-10 against the direct solve (T2 bars), and the
    FP64 form's update count against the per-set factors' (the same iteration
    up to rounding)."""
    from paper_1208_4093_gb300 import capi
    tr, g, pr = make(hms_ctx, case, prec, tol=1e-10, max_iter=2000)
    name, nx, ny, sx, sy, fixb = case
    p = loads(nx, ny, 7).reshape(-1)
    u_ref = direct.cholesky_solve(tr, tr.free * p)
    try:
        u, its = np.empty((1, tr.ndof)), np.zeros(1, np.int32)
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u, iters=its)
    finally:
        capi.hms_problem_destroy(pr)
    assert rel(u[0], u_ref) < (1e-8 if prec == 1 else 1e-9)
    fixed = fixb(nx, ny) if fixb else None
    ps = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, fixed=fixed, precision=prec, tol=1e-10, max_iter=2000)
    try:
        u2, its2 = np.empty((1, tr.ndof)), np.zeros(1, np.int32)
        capi.hms_solve(hms_ctx, ps, p.reshape(1, -1), u2, iters=its2)
    finally:
        capi.hms_problem_destroy(ps)
    assert abs(int(its[0]) - int(its2[0])) <= 1
    assert rel(u[0], u2[0]) < (1e-8 if prec == 1 else 1e-9)


def test_class_factors_deterministic(hms_ctx):
    from paper_1208_4093_gb300 import capi
    tr, g, pr = make(hms_ctx, CASES[3], 1, tol=1e-9, max_iter=500)
    p = loads(tr.nx, tr.ny, 2).reshape(1, -1)
    try:
        a, b = np.empty((1, tr.ndof)), np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p, a)
        capi.hms_solve(hms_ctx, pr, p, b)
    finally:
        capi.hms_problem_destroy(pr)
    assert np.array_equal(a, b)


def test_class_factors_rejections(hms_ctx):
    from paper_1208_4093_gb300 import capi
    from workloads import ea_lognormal
    bad = [dict(ea=ea_lognormal(32, 32, 1)), dict(relax_overlap=2), dict(mode_mask=0xFFF), dict(class_factors=2)]
    for kw in bad:
        args = dict(class_factors=1)
        args.update(kw)
        with pytest.raises(RuntimeError):
            capi.hms_problem_create(hms_ctx, 32, 32, 8, 8, **args)
        assert capi.hms_problem_estimate_bytes(hms_ctx, 32, 32, 8, 8, **args) == 0


@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
def test_class_estimate_equals_allocation(hms_ctx, prec):
    from paper_1208_4093_gb300 import capi
    kw = dict(precision=prec, class_factors=1, tol=1e-8, max_iter=100)
    est = capi.hms_problem_estimate_bytes(hms_ctx, 200, 150, 32, 32, **kw)
    pr = capi.hms_problem_create(hms_ctx, 200, 150, 32, 32, **kw)
    try:
        held = capi.hms_problem_device_bytes(pr)
    finally:
        capi.hms_problem_destroy(pr)
    # the estimate adds the scratch held during setup
    assert held < est < held + 64 * 2**20
    per_set = capi.hms_problem_estimate_bytes(hms_ctx, 200, 150, 32, 32, precision=prec, tol=1e-8, max_iter=100)
    assert est < per_set  # the class factors take far less than one factor per set


def test_class_factors_in_batches_and_clones(hms_ctx):
    """Problems with class factors (and a clone sharing them) solved together
    by hms_solve_batch equal their solo solves bit for bit, and the automatic
    engine choice falls back to the stream engine for them."""
    from paper_1208_4093_gb300 import capi
    specs = [(100, 80, 16, 16, 0), (131, 70, 32, 16, 1), (100, 80, 16, 16, 2)]
    prs = []
    for nx, ny, sx, sy, _ in specs[:2]:
        prs.append(capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, precision=1, tol=1e-9, max_iter=2000,
                                           class_factors=1))
    prs.append(capi.hms_problem_clone(hms_ctx, prs[0]))
    try:
        loads_ = [loads(nx, ny, seed).reshape(1, -1) for nx, ny, _, _, seed in specs]
        outs = [np.empty_like(p) for p in loads_]
        its = np.zeros(3, np.int32)
        capi.hms_solve_batch(hms_ctx, prs, loads_, outs, iters=its)
        for k, pr in enumerate(prs):
            solo = np.empty_like(loads_[k])
            it1 = np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr, loads_[k], solo, iters=it1)
            assert np.array_equal(solo, outs[k]), k
            assert int(it1[0]) == int(its[k])
            nx, ny = specs[k][:2]
            tr = truss.Truss(nx, ny)
            assert rel(outs[k][0], direct.cholesky_solve(tr, tr.free * loads_[k][0])) < 1e-8
    finally:
        for pr in prs:
            capi.hms_problem_destroy(pr)
