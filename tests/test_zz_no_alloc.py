"""The allocation-free residual entry point against hms_residual and the oracle.

hms_residual_noalloc is for callers that cannot allocate device memory while
they call (a busy device where cudaFree would synchronise it, or HBM already
committed).  It computes the same r = p - K u and sums as hms_residual, with
its per-CTA partial sums and completion counter in static device memory.  Two
calls in a row must both match hms_residual: the second one only does if the
first left the counter at zero.  Both are also checked against the oracle's
assembled K.  This file is named to be collected last, so that it also runs
after every other GPU test has used the context.
"""
import ctypes

import numpy as np
import pytest

from workloads import ea_lognormal, loads

pytestmark = pytest.mark.gpu

CASES = [
    # nx, ny, sx, sy, lognormal EA: ragged tiles in x and y, uniform and lognormal EA
    (300, 77, 32, 16, True),
    (67, 24, 16, 12, False),
    (1024, 1024, 64, 64, True),
]


def _problem(capi, ctx, nx, ny, sx, sy, lognormal, precision=None):
    ea = ea_lognormal(nx, ny, seed=5) if lognormal else None
    return capi.hms_problem_create(ctx, nx, ny, sx, sy, ea=ea,
                                   precision=capi.HMS_FP64 if precision is None else precision)


@pytest.mark.parametrize("nx,ny,sx,sy,lognormal", CASES)
def test_two_calls_match_hms_residual(hms_ctx, nx, ny, sx, sy, lognormal):
    import torch
    from paper_1208_4093_gb300 import capi
    pr = _problem(capi, hms_ctx, nx, ny, sx, sy, lognormal)
    try:
        dev = torch.device("cuda:0")
        p = torch.from_numpy(loads(nx, ny, seed=12).reshape(-1)).to(dev)
        u = torch.from_numpy(loads(nx, ny, seed=11).reshape(-1)).to(dev)
        r_ref = torch.empty_like(p)
        n_ref = torch.empty(3, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        capi.hms_residual(hms_ctx, pr, p, u, r_ref, n_ref)
        outs = []
        for _ in range(2):
            r = torch.full_like(p, float("nan"))
            nrm = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
            torch.cuda.synchronize()
            capi.hms_residual_noalloc(hms_ctx, pr, p, u, r, nrm)
            outs.append((r.cpu().numpy(), nrm.cpu().numpy()))
        rr, nr = r_ref.cpu().numpy(), n_ref.cpu().numpy()
        scale = np.abs(rr).max()
        # the oracle: K assembled bar by bar, constrained DOFs of u read as 0
        from oracle import truss
        tr = truss.Truss(nx, ny, ea_lognormal(nx, ny, seed=5) if lognormal else None)
        pn, un = p.cpu().numpy(), u.cpu().numpy()
        ro = tr.residual(pn, un)
        uf = tr.free * un
        no = np.array([np.abs(ro).sum(), ro @ ro, uf @ (tr.free * pn + ro)])
        for r, nrm in outs:
            np.testing.assert_allclose(r, rr, rtol=1e-13, atol=1e-13 * scale)
            np.testing.assert_allclose(nrm, nr, rtol=1e-12)
            assert np.abs(r - ro).max() <= 1e-13 * np.abs(ro).max()
            np.testing.assert_allclose(nrm, no, rtol=1e-11)
        # inputs are read in place and left unchanged
        assert torch.equal(p.cpu(), torch.from_numpy(loads(nx, ny, seed=12).reshape(-1)))
    finally:
        capi.hms_problem_destroy(pr)


def test_rejects_host_misaligned_and_aliased(hms_ctx):
    """Argument checks run on the host before any launch."""
    import torch
    from paper_1208_4093_gb300 import capi
    nx, ny = 67, 24
    pr = _problem(capi, hms_ctx, nx, ny, 16, 12, False)
    try:
        dev = torch.device("cuda:0")
        p = torch.zeros(2 * nx * ny + 2, dtype=torch.float64, device=dev)
        u = torch.zeros_like(p)
        r = torch.zeros_like(p)
        host = np.zeros(2 * nx * ny, np.float64)
        f = capi.lib().hms_residual_noalloc
        assert f(pr, host.ctypes.data, u.data_ptr(), r.data_ptr(), None) == capi.HMS_ERR_ARG
        assert f(pr, p.data_ptr() + 8, u.data_ptr(), r.data_ptr(), None) == capi.HMS_ERR_ARG
        assert f(pr, p.data_ptr(), u.data_ptr(), u.data_ptr(), None) == capi.HMS_ERR_ARG
        # r overlapping u or p at an offset (16-byte aligned, so only the overlap is wrong)
        assert f(pr, p.data_ptr(), u.data_ptr(), u.data_ptr() + 16, None) == capi.HMS_ERR_ARG
        assert f(pr, p.data_ptr() + 16, u.data_ptr(), p.data_ptr(), None) == capi.HMS_ERR_ARG
        assert f(pr, p.data_ptr(), u.data_ptr(), r.data_ptr(), r.data_ptr() + 4) == capi.HMS_ERR_ARG
        assert f(pr, None, u.data_ptr(), r.data_ptr(), None) == capi.HMS_ERR_ARG
        with pytest.raises(ValueError):
            capi.hms_residual_noalloc(hms_ctx, pr, host, host, host.copy())
        # a valid call still works after the rejected ones
        capi.hms_residual_noalloc(hms_ctx, pr, p[:2 * nx * ny], u[:2 * nx * ny], r[:2 * nx * ny])
        torch.cuda.synchronize()
        assert float(r.abs().sum()) == 0.0
    finally:
        capi.hms_problem_destroy(pr)


def test_rejects_lattice_beyond_static_scratch(hms_ctx):
    """1024 x 4104 nodes need 32 * 513 = 16416 tiles of 32 x 8 > 16384."""
    import torch
    from paper_1208_4093_gb300 import capi
    nx, ny = 1024, 4104
    pr = capi.hms_problem_create(hms_ctx, nx, ny, 64, 64, precision=capi.HMS_MIXED)
    try:
        v = torch.zeros(2 * nx * ny, dtype=torch.float64, device="cuda:0")
        r = torch.empty_like(v)
        with pytest.raises(capi.HmsError) as e:
            capi.hms_residual_noalloc(hms_ctx, pr, v, v, r)
        assert e.value.status == capi.HMS_ERR_ARG
        assert "16416" in str(e.value) and "hms_residual" in str(e.value)
    finally:
        capi.hms_problem_destroy(pr)
