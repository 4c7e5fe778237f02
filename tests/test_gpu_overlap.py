"""Extended relaxation regions (Sec. 2.2, the region around a set in Fig. 1)
through the C ABI against the oracle.

With relax_overlap = e every set relaxes together with the nodes within e
nodes of its tile (clipped to the lattice), all other DOFs held, and keeps its
own nodes' part of the increment as its mode.  The relaxation step is compared
element by element with ``oracle.hms.LocalFactors(overlap=e)``; whole solves
with the oracle's iteration (update counts) and the direct solve.  Tolerances
as in test_gpu_parity.py: FP64 local solves 1e-11 (local condition numbers
<= 1e4 here), FP32 relaxation 2e-5, converged displacement 1e-9 (FP64) and
1e-8 (mixed).
"""
import numpy as np
import pytest

from oracle import direct, hms, truss
from workloads import ea_lognormal, loads

pytestmark = pytest.mark.gpu

# name, nx, ny, sx, sy, lognormal EA, overlap
CASES = [
    ("ragged_e1", 37, 29, 8, 6, True, 1),
    ("ragged_e3", 37, 29, 8, 6, True, 3),
    ("odd_rows_e2", 20, 13, 7, 5, False, 2),
    ("wide_e4", 67, 24, 32, 12, True, 4),
    ("one_row_sets_e2", 16, 9, 8, 1, False, 2),
]
# regions wider than 64 nodes: mixed path only
WIDE = [("region80_e8", 100, 30, 64, 10, True, 8)]
PRECS = [0, 1]


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    n = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (n if n > 0 else 1.0)


def make(ctx, case, prec, tol=1e-11, max_iter=800, **kw):
    from paper_1208_4093_gb300 import capi
    name, nx, ny, sx, sy, ln, e = case
    ea = ea_lognormal(nx, ny, 17) if ln else None
    tr = truss.Truss(nx, ny, ea)
    g = hms.SetGrid(nx, ny, sx, sy)
    p = loads(nx, ny, 5).reshape(-1)
    pr = capi.hms_problem_create(ctx, nx, ny, sx, sy, ea=ea, precision=prec, tol=tol, max_iter=max_iter,
                                 relax_overlap=e, **kw)
    return tr, g, p, pr


@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_overlap_relax_step(hms_ctx, case, prec):
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = make(hms_ctx, case, prec)
    try:
        u = tr.free * np.random.default_rng(3).standard_normal(tr.ndof)
        r = tr.residual(tr.free * p, u)
        dl, P = np.empty(tr.ndof), np.empty(9 * g.M)
        capi.hms_relax(hms_ctx, pr, r, dl, P)
        do = hms.LocalFactors(tr, g, overlap=case[6]).relax(r)
        assert rel(dl, do) < (2e-5 if prec == 1 else 1e-11)
        assert np.all(dl[~tr.free] == 0)
        Po = hms.modes(tr, g, dl).T @ r
        assert rel(P, Po) < 1e-12
    finally:
        capi.hms_problem_destroy(pr)


@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_overlap_full_solve(hms_ctx, case, prec):
    """Converged displacement against the direct solve; FP64 update counts
    against the oracle's iteration with the same regions."""
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = make(hms_ctx, case, prec)
    try:
        u = np.empty((1, tr.ndof))
        its = np.zeros(1, np.int32)
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u, iters=its)
        u_ref = direct.cholesky_solve(tr, tr.free * p)
        assert rel(u[0], u_ref) < (1e-8 if prec == 1 else 1e-9)
        if prec == 0:
            res = hms.solve(tr, g, p, 1e-11, 800, factors=hms.LocalFactors(tr, g, overlap=case[6]))
            assert abs(int(its[0]) - res.iterations) <= 1
    finally:
        capi.hms_problem_destroy(pr)


def test_overlap_reduces_updates_and_covering_region_is_direct(hms_ctx):
    """Fewer updates with a larger region (Sec. 2.2); grown over the whole
    lattice, one update is the direct solve."""
    from paper_1208_4093_gb300 import capi
    nx, ny = 24, 20
    tr = truss.Truss(nx, ny)
    p = loads(nx, ny, 3).reshape(1, -1)
    nir = []
    for e in (0, 1, 4, 24):
        pr = capi.hms_problem_create(hms_ctx, nx, ny, 8, 8, tol=1e-11, max_iter=500, relax_overlap=e)
        try:
            u = np.empty_like(p)
            its = np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr, p, u, iters=its)
            nir.append(int(its[0]))
        finally:
            capi.hms_problem_destroy(pr)
    assert nir[0] > nir[1] > nir[2] > nir[3] == 1, nir
    assert rel(u[0], direct.cholesky_solve(tr, tr.free * p[0])) < 1e-11


def test_overlap_launch_shapes_and_batch_agree(hms_ctx):
    """The relaxation's CTA sizes give the same bits with overlap, and so do
    the lockstep batch and the solo solve."""
    from paper_1208_4093_gb300 import capi
    nx, ny, e = 48, 40, 2
    ea = ea_lognormal(nx, ny, 4)
    p = loads(nx, ny, 8).reshape(1, -1)
    outs = []
    for nt in (64, 128, 256):
        pr = capi.hms_problem_create(hms_ctx, nx, ny, 16, 16, ea=ea, precision=1, tol=1e-10, max_iter=800,
                                     relax_overlap=e, relax_threads=nt, relax_copies=1, coarse_factor=4)
        try:
            u = np.empty_like(p)
            capi.hms_solve(hms_ctx, pr, p, u)
            outs.append(u)
        finally:
            capi.hms_problem_destroy(pr)
    assert all(np.array_equal(outs[0], o) for o in outs[1:])
    a = capi.hms_problem_create(hms_ctx, nx, ny, 16, 16, ea=ea, precision=1, tol=1e-10, max_iter=800,
                                relax_overlap=e, coarse_factor=4)
    b = capi.hms_problem_create(hms_ctx, 30, 22, 8, 8, precision=1, tol=1e-10, max_iter=800, relax_overlap=1,
                                coarse_factor=4)
    try:
        q = loads(30, 22, 2).reshape(1, -1)
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_LOCKSTEP)
        ua, ub = np.empty_like(p), np.empty_like(q)
        capi.hms_solve_batch(hms_ctx, [a, b], [p, q], [ua, ub])
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_AUTO)
        sa, sb = np.empty_like(p), np.empty_like(q)
        capi.hms_solve(hms_ctx, a, p, sa)
        capi.hms_solve(hms_ctx, b, q, sb)
        assert np.array_equal(ua, sa) and np.array_equal(ub, sb)
        assert np.array_equal(ua, outs[0])
    finally:
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_AUTO)
        capi.hms_problem_destroy(a)
        capi.hms_problem_destroy(b)


def test_overlap_rejections(hms_ctx):
    from paper_1208_4093_gb300 import capi
    for kw in (dict(relax_overlap=-1), dict(relax_overlap=25), dict(relax_overlap=1, relax_copies=2),
               dict(relax_overlap=17, precision=0)):
        with pytest.raises(capi.HmsError) as e:
            capi.hms_problem_create(hms_ctx, 96, 40, 32, 16, **kw)
        assert e.value.status == capi.HMS_ERR_ARG, kw
    # the grown tile is clipped to the lattice: 40 nodes wide is fine at any overlap
    pr = capi.hms_problem_create(hms_ctx, 40, 24, 32, 8, relax_overlap=40)
    capi.hms_problem_destroy(pr)
    # up to 80 nodes on the mixed path (FP32 factors), at most 64 with FP64 ones
    pr = capi.hms_problem_create(hms_ctx, 96, 40, 32, 16, relax_overlap=24, precision=1)
    capi.hms_problem_destroy(pr)


def test_overlap_after_the_same_set_shape_without(hms_ctx):
    """The launch-shape tuner keeps its choice per set shape, precision and
    overlap: a shape tuned without overlap (where two copies per matrix may
    win) must not hand that choice to a problem with overlap."""
    from paper_1208_4093_gb300 import capi
    nx, ny = 52, 40
    p = loads(nx, ny, 6).reshape(1, -1)
    a = capi.hms_problem_create(hms_ctx, nx, ny, 26, 20, tol=1e-10, max_iter=500, relax_copies=2)
    b = capi.hms_problem_create(hms_ctx, nx, ny, 26, 20, tol=1e-10, max_iter=500)
    c = capi.hms_problem_create(hms_ctx, nx, ny, 26, 20, tol=1e-10, max_iter=500, relax_overlap=3)
    try:
        assert capi.hms_problem_relax_copies(c) == 1
        ua, uc = np.empty_like(p), np.empty_like(p)
        capi.hms_solve(hms_ctx, a, p, ua)
        capi.hms_solve(hms_ctx, c, p, uc)
        tr = truss.Truss(nx, ny)
        ref = direct.cholesky_solve(tr, tr.free * p[0])
        assert rel(uc[0], ref) < 1e-9 and rel(ua[0], ref) < 1e-9
        assert capi.hms_problem_relax_copies(b) in (1, 2)
    finally:
        for q in (a, b, c):
            capi.hms_problem_destroy(q)


@pytest.mark.parametrize("case", WIDE, ids=lambda c: c[0])
def test_overlap_regions_wider_than_64_nodes_mixed(hms_ctx, case):
    """Regions up to 80 nodes wide on the mixed path: the relaxation step
    against the oracle and the converged displacement against the direct solve."""
    from paper_1208_4093_gb300 import capi
    tr, g, p, pr = make(hms_ctx, case, 1)
    try:
        u = tr.free * np.random.default_rng(4).standard_normal(tr.ndof)
        r = tr.residual(tr.free * p, u)
        dl, P = np.empty(tr.ndof), np.empty(9 * g.M)
        capi.hms_relax(hms_ctx, pr, r, dl, P)
        assert rel(dl, hms.LocalFactors(tr, g, overlap=case[6]).relax(r)) < 2e-5
        us = np.empty((1, tr.ndof))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), us)
        assert rel(us[0], direct.cholesky_solve(tr, tr.free * p)) < 1e-8
    finally:
        capi.hms_problem_destroy(pr)
    with pytest.raises(capi.HmsError):
        make(hms_ctx, case, 0)
