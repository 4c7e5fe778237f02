"""The rest of the C-ABI boundary: reactions (K u at every DOF), the mode
mask, the history switch, the refinement counter and the timeout path.

Expected values come from the oracle: ``oracle.truss.Truss.reactions`` (K
assembled bar by bar) and ``oracle.hms.solve(..., mode_mask=...)`` (the
iteration with the same incremental modes left out of Eq. 3).
"""
import numpy as np
import pytest

from workloads import ea_lognormal, loads

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.mark.parametrize("nx,ny,lognormal", [(37, 29, True), (64, 48, False), (130, 17, True)])
def test_reactions_match_oracle(hms_ctx, nx, ny, lognormal):
    """K u at every DOF (constrained ones included) against the oracle's
    assembled K, for a random u (nonzero on constrained DOFs too, which the
    library must read as 0)."""
    from oracle import truss
    from paper_1208_4093_gb300 import capi
    ea = ea_lognormal(nx, ny, 3) if lognormal else None
    pr = capi.hms_problem_create(hms_ctx, nx, ny, 16, 16, ea=ea)
    try:
        u = loads(nx, ny, 21).reshape(-1)
        f = np.empty_like(u)
        capi.hms_reactions(hms_ctx, pr, u, f)
    finally:
        capi.hms_problem_destroy(pr)
    tr = truss.Truss(nx, ny, ea)
    ref = tr.reactions(u)
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()
    # the constrained DOFs carry support forces (not zeroed like the residual)
    fixed = ~tr.free
    assert np.abs(f[fixed]).max() > 0.0


def test_reactions_balance_loads_at_convergence(hms_ctx):
    """At a converged solution the support reactions balance the applied loads
    in force and in moment (the bar forces of any u are self-equilibrated:
    1^T K u = 0 and the moment of K u about the origin is 0)."""
    from oracle import truss
    from paper_1208_4093_gb300 import capi
    nx, ny = 96, 80
    ea = ea_lognormal(nx, ny, 8)
    tr = truss.Truss(nx, ny, ea)
    p = tr.free * loads(nx, ny, 9).reshape(-1)
    pr = capi.hms_problem_create(hms_ctx, nx, ny, 32, 16, ea=ea, tol=1e-13, max_iter=3000)
    try:
        u = np.empty((1, p.size))
        capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u)
        f = np.empty_like(p)
        capi.hms_reactions(hms_ctx, pr, u[0], f)
    finally:
        capi.hms_problem_destroy(pr)
    fixed = ~tr.free
    x = np.repeat(tr.x.reshape(-1), 2)
    y = np.repeat(tr.y.reshape(-1), 2)
    isx = np.arange(p.size) % 2 == 0
    reac = np.where(fixed, f, 0.0)
    scale = np.abs(p).sum()
    for comp in (isx, ~isx):
        assert abs(reac[comp].sum() + p[comp].sum()) <= 1e-10 * scale
    mom = lambda v: (x[~isx] * v[~isx]).sum() - (y[isx] * v[isx]).sum()  # noqa: E731
    assert abs(mom(reac) + mom(p)) <= 1e-10 * scale * max(nx, ny)
    # on the free DOFs K u equals the load to the solve's tolerance
    assert np.abs(f[tr.free] - p[tr.free]).sum() <= 1e-12 * scale


def test_reactions_arguments(hms_ctx):
    import torch
    from paper_1208_4093_gb300 import capi
    nx, ny = 20, 12
    pr = capi.hms_problem_create(hms_ctx, nx, ny, 10, 6)
    try:
        f = capi.lib().hms_reactions
        v = torch.zeros(2 * nx * ny + 2, dtype=torch.float64, device="cuda:0")
        assert f(pr, None, v.data_ptr(), capi.HMS_MEM_DEVICE) == capi.HMS_ERR_ARG
        assert f(pr, v.data_ptr(), v.data_ptr() + 16, capi.HMS_MEM_DEVICE) == capi.HMS_ERR_ARG
        assert f(pr, v.data_ptr(), v.data_ptr(), 7) == capi.HMS_ERR_ARG
    finally:
        capi.hms_problem_destroy(pr)


@pytest.mark.parametrize("mask", [0x03F, 0x07F, 0x1C3, 0x1FC])
@pytest.mark.parametrize("precision", [0, 1])
def test_mode_mask_trajectory_matches_oracle(hms_ctx, mask, precision):
    """Modes left out of the upper-level correction get a = 0: the iterates
    equal the oracle's iteration with the same modes (T1 per update; the mixed
    path within the FP32 relaxation's reach)."""
    from oracle import hms, truss
    from paper_1208_4093_gb300 import capi
    nx, ny, sx, sy = 40, 33, 12, 10
    ea = ea_lognormal(nx, ny, 4)
    tr = truss.Truss(nx, ny, ea)
    grid = hms.SetGrid(nx, ny, sx, sy)
    p = tr.free * loads(nx, ny, 5).reshape(-1)
    steps = 4
    ref = hms.solve(tr, grid, p, 0.0, steps, mode_mask=mask, keep_iterates=True).iterates
    for k in (1, steps):
        pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, ea=ea, precision=precision, tol=0.0, max_iter=k,
                                     mode_mask=mask)
        try:
            u = np.empty((1, p.size))
            capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u, allow_no_convergence=True)
        finally:
            capi.hms_problem_destroy(pr)
        assert rel(u[0], ref[k - 1]) < (1e-9 if precision == 0 else 1e-4), (mask, k)


def test_mode_mask_rejects_bits_above_twelve(hms_ctx):
    """Bits 0-8: the displacement-controlled modes; 9-11: the force-controlled
    ones (q = 12, tests/test_gpu_force.py); nothing above."""
    from paper_1208_4093_gb300 import capi
    with pytest.raises(capi.HmsError) as e:
        capi.hms_problem_create(hms_ctx, 20, 20, 10, 10, mode_mask=0x1FFF)
    assert e.value.status == capi.HMS_ERR_ARG
    pr = capi.hms_problem_create(hms_ctx, 20, 20, 10, 10, mode_mask=0x3FF)
    capi.hms_problem_destroy(pr)


def test_relax_overlap_overflow_rejected(hms_ctx):
    """set_sx + 2 relax_overlap beyond the int range is an argument error,
    not a wrapped-around small width."""
    from paper_1208_4093_gb300 import capi
    for ov in (2 ** 31 - 1, 2 ** 30):
        with pytest.raises(capi.HmsError) as e:
            capi.hms_problem_create(hms_ctx, 200, 40, 16, 16, precision=capi.HMS_MIXED, relax_overlap=ov)
        assert e.value.status == capi.HMS_ERR_ARG
        assert capi.hms_problem_estimate_bytes(hms_ctx, 200, 40, 16, 16, precision=capi.HMS_MIXED,
                                               relax_overlap=ov) == 0


def test_record_history_switch(hms_ctx):
    from paper_1208_4093_gb300 import capi
    nx, ny = 48, 40
    p = loads(nx, ny, 2).reshape(1, -1)
    out = {}
    for rec in (1, 0):
        pr = capi.hms_problem_create(hms_ctx, nx, ny, 16, 16, tol=1e-10, max_iter=500, record_history=rec)
        try:
            u = np.empty_like(p)
            hist = np.zeros((1, 501, 3))
            its = np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr, p, u, hist=hist, iters=its)
            out[rec] = (u, hist, int(its[0]), capi.hms_problem_device_bytes(pr))
        finally:
            capi.hms_problem_destroy(pr)
    u1, h1, n1, b1 = out[1]
    u0, h0, n0, b0 = out[0]
    assert np.array_equal(u0, u1) and n0 == n1
    assert np.isfinite(h1[0, :n1 + 1]).all() and np.isnan(h0).all()
    assert b1 - b0 == 3 * 8 * 501


def test_refine_cap_hits_counter(hms_ctx):
    """With two solves per update the FP32 factor's first solve never meets the
    1e-14 refinement criterion, so every update uses its last solve; with
    eight, refinement converges earlier in (nearly) every update."""
    from paper_1208_4093_gb300 import capi
    nx, ny = 64, 64
    p = loads(nx, ny, 0).reshape(1, -1)
    hits = {}
    for ns in (1, 2, 8):
        pr = capi.hms_problem_create(hms_ctx, nx, ny, 16, 16, tol=1e-8, max_iter=1000, coarse_solves=ns,
                                     coarse_factor=4)
        try:
            u = np.empty_like(p)
            its = np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr, p, u, iters=its)
            hits[ns] = (capi.hms_problem_refine_cap_hits(pr), int(its[0]))
        finally:
            capi.hms_problem_destroy(pr)
    assert hits[1][0] == 0
    assert hits[2][0] == hits[2][1]
    assert hits[8][0] < hits[2][0]


@pytest.mark.parametrize("precision", [0, 1])
def test_relaxation_timeout_is_reported_and_recovers(hms_ctx, precision):
    """The relaxation's first copy wait made to give up at once: the kernel
    drains its own copies, raises the flag, and the call returns
    HMS_ERR_TIMEOUT; with the usual bound restored the same problem solves
    normally."""
    from oracle import hms, truss
    from paper_1208_4093_gb300 import capi
    nx, ny, sx, sy = 64, 40, 16, 20
    tr = truss.Truss(nx, ny)
    p = tr.free * loads(nx, ny, 7).reshape(-1)
    pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, precision=precision, tol=1e-10, max_iter=3,
                                 relax_threads=128)
    try:
        capi.hms_problem_set_relax_wait_limit(hms_ctx, pr, 0)
        r = p.copy()
        d = np.empty_like(r)
        P = np.empty(9 * 4 * 2)
        with pytest.raises(capi.HmsError) as e:
            capi.hms_relax(hms_ctx, pr, r, d, P)
        assert e.value.status == capi.HMS_ERR_TIMEOUT
        u = np.empty((1, p.size))
        with pytest.raises(capi.HmsError) as e:
            capi.hms_solve(hms_ctx, pr, p.reshape(1, -1), u, allow_no_convergence=True)
        assert e.value.status == capi.HMS_ERR_TIMEOUT
        capi.hms_problem_set_relax_wait_limit(hms_ctx, pr, -1)
        capi.hms_relax(hms_ctx, pr, r, d, P)
        ref = hms.LocalFactors(tr, hms.SetGrid(nx, ny, sx, sy)).relax(p)
        assert rel(d, ref) < (1e-11 if precision == 0 else 2e-5)
    finally:
        capi.hms_problem_destroy(pr)
