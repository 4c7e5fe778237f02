"""The relaxation on the balanced schedule (relax_balance = 2) against the
oracle and against one CTA per set.

One persistent CTA per SM runs an equal share of all sets' substitution
steps; a set cut between two CTAs hands its state over through device memory
(y_j or x_j) and a per-set flag.  Every op's arithmetic is that of the
one-CTA-per-set kernel, so delta (Eq. 13) and P (Eq. 7) must agree bit for
bit, and with the oracle's per-set local solves (Eq. 12) at the tolerances
of test_gpu_parity: FP64 1e-11, FP32 2e-5.  The lattices have more sets than
a GB300 has SMs (152), so sets are cut between CTAs, in the forward and in
the backward pass.
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


# name, nx, ny, sx, sy: 15 x 14 sets; the same with a ragged last row and
# column of sets; 13 x 13 sets (the share per SM just over one set)
CASES = [("sets210", 120, 112, 8, 8), ("sets210_ragged", 118, 110, 8, 8), ("sets169", 104, 104, 8, 8)]
PRECS = [0, 1]


def pair(ctx, nx, ny, sx, sy, prec, **kw):
    from paper_1208_4093_gb300 import capi
    a = capi.hms_problem_create(ctx, nx, ny, sx, sy, precision=prec, relax_balance=2, **kw)
    try:
        b = capi.hms_problem_create(ctx, nx, ny, sx, sy, precision=prec, relax_balance=1, relax_threads=256,
                                    relax_copies=1, **kw)
    except Exception:
        capi.hms_problem_destroy(a)
        raise
    assert capi.hms_problem_relax_balanced(a) == 1
    assert capi.hms_problem_relax_balanced(b) == 0
    return a, b


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
def test_balanced_relax_step(hms_ctx, case, prec):
    from paper_1208_4093_gb300 import capi
    _, nx, ny, sx, sy = case
    tr = truss.Truss(nx, ny)
    g = hms.SetGrid(nx, ny, sx, sy)
    a, b = pair(hms_ctx, nx, ny, sx, sy, prec, tol=1e-10, max_iter=10)
    try:
        for seed in (3, 4):
            u = tr.free * np.random.default_rng(seed).standard_normal(tr.ndof)
            r = tr.residual(tr.free * loads(nx, ny, seed).reshape(-1), u)
            da, Pa = np.empty(tr.ndof), np.empty(9 * g.M)
            db, Pb = np.empty(tr.ndof), np.empty(9 * g.M)
            capi.hms_relax(hms_ctx, a, r, da, Pa)
            capi.hms_relax(hms_ctx, b, r, db, Pb)
            assert np.array_equal(da, db)
            assert np.array_equal(Pa, Pb)
            do = hms.LocalFactors(tr, g).relax(r)
            assert rel(da, do) < (2e-5 if prec == 1 else 1e-11)
            assert rel(Pa, hms.modes(tr, g, da).T @ r) < 1e-12
            # the same problem again: the set flags were reset by the launch before
            capi.hms_relax(hms_ctx, a, r, da, Pa)
            assert np.array_equal(da, db) and np.array_equal(Pa, Pb)
    finally:
        capi.hms_problem_destroy(a)
        capi.hms_problem_destroy(b)


@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
def test_balanced_solve_matches_per_set_and_direct(hms_ctx, prec):
    """Whole solves (the iteration captured in CUDA graphs with the
    cooperative launch) equal bit for bit; both against the direct solve."""
    from paper_1208_4093_gb300 import capi
    _, nx, ny, sx, sy = CASES[1]
    tr = truss.Truss(nx, ny)
    p = loads(nx, ny, 5).reshape(1, -1)
    a, b = pair(hms_ctx, nx, ny, sx, sy, prec, tol=1e-10, max_iter=3000)
    c = capi.hms_problem_clone(hms_ctx, a)
    try:
        outs, its = [], []
        for pr in (a, b, c):
            u, it = np.empty_like(p), np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr, p, u, iters=it)
            outs.append(u)
            its.append(int(it[0]))
        assert capi.hms_problem_relax_balanced(c) == 1
    finally:
        for pr in (a, b, c):
            capi.hms_problem_destroy(pr)
    assert its[0] == its[1] == its[2]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])
    assert rel(outs[0][0], direct.cholesky_solve(tr, tr.free * p[0])) < (1e-8 if prec == 1 else 1e-9)


@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
def test_balanced_relax_benchmark_lattice(hms_ctx, prec):
    """The 1024^2 lognormal lattice (16 x 16 sets of 64 x 64 nodes: 256 sets
    on 152 SMs, each SM 1.68 sets' work): bitwise the one-CTA-per-set result."""
    torch = pytest.importorskip("torch")
    from paper_1208_4093_gb300 import capi
    from workloads import CASES as W
    c = W["lattice1024_lognormal_fp64"]
    ea = c.ea_array()
    kw = dict(ea=ea, tol=1e-8, max_iter=10)
    a, b = pair(hms_ctx, c.nx, c.ny, c.sx, c.sy, prec, **kw)
    try:
        r = torch.from_numpy(c.load_array().reshape(-1)).cuda()
        outs = []
        for pr in (a, b):
            d = torch.empty_like(r)
            P = torch.empty(9 * 256, dtype=torch.float64, device="cuda")
            capi.hms_relax(hms_ctx, pr, r, d, P)
            outs.append((d, P))
        torch.cuda.synchronize()
        assert torch.equal(outs[0][0], outs[1][0])
        assert torch.equal(outs[0][1], outs[1][1])
        assert torch.count_nonzero(outs[0][0]).item() > 0
    finally:
        capi.hms_problem_destroy(a)
        capi.hms_problem_destroy(b)


def test_balanced_timeout_is_reported_and_recovers(hms_ctx):
    """Every CTA's first copy wait made to give up: the launch drains its
    copies and reports HMS_ERR_TIMEOUT; with the usual bound the same problem
    relaxes correctly (no set flag left raised)."""
    from paper_1208_4093_gb300 import capi
    _, nx, ny, sx, sy = CASES[0]
    tr = truss.Truss(nx, ny)
    g = hms.SetGrid(nx, ny, sx, sy)
    p = tr.free * loads(nx, ny, 7).reshape(-1)
    pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, tol=1e-10, max_iter=3, relax_balance=2)
    try:
        capi.hms_problem_set_relax_wait_limit(hms_ctx, pr, 0)
        d, P = np.empty_like(p), np.empty(9 * g.M)
        with pytest.raises(capi.HmsError) as e:
            capi.hms_relax(hms_ctx, pr, p, d, P)
        assert e.value.status == capi.HMS_ERR_TIMEOUT
        capi.hms_problem_set_relax_wait_limit(hms_ctx, pr, -1)
        capi.hms_relax(hms_ctx, pr, p, d, P)
        assert rel(d, hms.LocalFactors(tr, g).relax(p)) < 1e-11
    finally:
        capi.hms_problem_destroy(pr)


def test_balanced_rejections(hms_ctx):
    from paper_1208_4093_gb300 import capi
    bad = [
        dict(nx=64, ny=64, sx=16, sy=16),                      # 16 sets: fewer than the SMs
        dict(nx=120, ny=112, sx=8, sy=8, relax_overlap=2),
        dict(nx=120, ny=112, sx=8, sy=8, relax_threads=128),
        dict(nx=120, ny=112, sx=8, sy=8, relax_copies=2),
        dict(nx=120, ny=112, sx=8, sy=8, class_factors=1),
    ]
    for kw in bad:
        nx, ny, sx, sy = kw.pop("nx"), kw.pop("ny"), kw.pop("sx"), kw.pop("sy")
        with pytest.raises(RuntimeError):
            capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, relax_balance=2, **kw)
    with pytest.raises(RuntimeError):
        capi.hms_problem_create(hms_ctx, 120, 112, 8, 8, relax_balance=3)
    assert capi.hms_problem_estimate_bytes(hms_ctx, 120, 112, 8, 8, relax_balance=3) == 0


@pytest.mark.parametrize("prec", PRECS, ids=["fp64", "mixed"])
def test_balanced_automatic_choice_is_cached(hms_ctx, prec):
    """relax_balance = 0 times the schedule with the CTA sizes; the second
    problem of the same shape takes the context's cached choice (schedule
    included) and both relax bit for bit like one CTA per set."""
    from paper_1208_4093_gb300 import capi
    _, nx, ny, sx, sy = CASES[0]
    tr = truss.Truss(nx, ny)
    g = hms.SetGrid(nx, ny, sx, sy)
    r = tr.free * loads(nx, ny, 9).reshape(-1)
    prs = [capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, precision=prec, relax_balance=0) for _ in range(2)]
    prs.append(capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, precision=prec, relax_balance=1,
                                       relax_threads=256, relax_copies=1))
    try:
        shapes = [(capi.hms_problem_relax_threads(p), capi.hms_problem_relax_copies(p),
                   capi.hms_problem_relax_balanced(p)) for p in prs[:2]]
        assert shapes[0] == shapes[1]
        assert shapes[0][1] in (1, 2) and shapes[0][2] in (0, 1)
        outs = []
        for p in prs:
            d, P = np.empty_like(r), np.empty(9 * g.M)
            capi.hms_relax(hms_ctx, p, r, d, P)
            outs.append((d, P))
        for d, P in outs[:2]:
            assert np.array_equal(d, outs[2][0]) and np.array_equal(P, outs[2][1])
    finally:
        for p in prs:
            capi.hms_problem_destroy(p)
