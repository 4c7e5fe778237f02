"""Batched uneven lattices: hms_solve_batch against solo solves and the oracle.

Lattices of different shapes and load-vector counts (the batched-lattice
generator of workloads/, 32 x 32-node sets with ragged edge sets, mixed
precision) are solved together.  Every lattice's result must equal its solo
hms_solve (the kernels of one problem are deterministic and share nothing with
the others), and the small ones must match the direct solve of the oracle
within the mixed path's 1e-8.
"""
import numpy as np
import pytest

from oracle import direct, truss
from workloads import batched_lattices

pytestmark = pytest.mark.gpu

TOL = 1e-9


@pytest.fixture(scope="module")
def batch(hms_ctx):
    from paper_1208_4093_gb300 import capi
    lats = batched_lattices(count=10, seed=11, side_min=8, side_max=96, nrhs_max=3)
    prs = [capi.hms_problem_create(hms_ctx, l.nx, l.ny, 32, 32, precision=capi.HMS_MIXED, tol=TOL,
                                   max_iter=4000) for l in lats]
    yield lats, prs
    for pr in prs:
        capi.hms_problem_destroy(pr)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_batch_equals_solo_and_oracle(hms_ctx, batch):
    from paper_1208_4093_gb300 import capi
    lats, prs = batch
    loads = [l.load_array() for l in lats]
    outs = [np.empty_like(p) for p in loads]
    its = np.zeros(sum(l.nrhs for l in lats), np.int32)
    capi.hms_solve_batch(hms_ctx, prs, loads, outs, iters=its)
    k = 0
    for l, pr, p, u in zip(lats, prs, loads, outs):
        solo = np.empty_like(p)
        sits = np.zeros(l.nrhs, np.int32)
        capi.hms_solve(hms_ctx, pr, p, solo, iters=sits)
        assert np.array_equal(u, solo), (l.nx, l.ny)
        assert np.array_equal(its[k:k + l.nrhs], sits)
        k += l.nrhs
        if l.nx * l.ny <= 4000:
            tr = truss.Truss(l.nx, l.ny)
            for r in range(l.nrhs):
                ref = direct.cholesky_solve(tr, tr.free * p[r])
                assert rel(u[r], ref) < 1e-8, (l.nx, l.ny, r)


def test_batch_device_tensors_match_host(hms_ctx, batch):
    import torch
    from paper_1208_4093_gb300 import capi
    lats, prs = batch
    sub = list(range(0, len(lats), 3))
    loads = [lats[i].load_array() for i in sub]
    host = [np.empty_like(p) for p in loads]
    capi.hms_solve_batch(hms_ctx, [prs[i] for i in sub], loads, host)
    dl = [torch.from_numpy(p).cuda() for p in loads]
    du = [torch.empty_like(t) for t in dl]
    torch.cuda.synchronize()
    capi.hms_solve_batch(hms_ctx, [prs[i] for i in sub], dl, du)
    torch.cuda.synchronize()
    for h, d in zip(host, du):
        assert np.array_equal(h, d.cpu().numpy())


def test_batch_rejects_duplicates_and_foreign_problems(hms_ctx, batch):
    from paper_1208_4093_gb300 import capi
    lats, prs = batch
    p = lats[0].load_array()
    with pytest.raises(capi.HmsError) as e:
        capi.hms_solve_batch(hms_ctx, [prs[0], prs[0]], [p, p], [np.empty_like(p), np.empty_like(p)])
    assert e.value.status == capi.HMS_ERR_ARG
    other = capi.hms_context_create(0)
    try:
        with pytest.raises(capi.HmsError) as e:
            capi.hms_solve_batch(other, [prs[0]], [p], [np.empty_like(p)])
        assert e.value.status == capi.HMS_ERR_ARG
    finally:
        capi.hms_context_destroy(other)
    # an empty batch is a no-op
    capi.hms_solve_batch(hms_ctx, [], [], [])


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_lockstep_equals_streams_and_solo(hms_ctx, prec):
    """The lockstep engine (one launch per step over a work list of every
    running problem's tiles) gives the stream engine's and the solo solves'
    bits, iteration counts included; lattices finish at different rounds and
    load vectors restart inside the batch."""
    from paper_1208_4093_gb300 import capi
    lats = batched_lattices(count=12, seed=13, side_min=8, side_max=160, nrhs_max=3)
    prs = [capi.hms_problem_create(hms_ctx, l.nx, l.ny, 32, 32, precision=prec, tol=TOL, max_iter=4000,
                                   coarse_factor=4) for l in lats]
    try:
        loads = [l.load_array() for l in lats]
        nrhs = sum(l.nrhs for l in lats)
        res = {}
        for mode in (capi.HMS_BATCH_LOCKSTEP, capi.HMS_BATCH_STREAMS):
            capi.hms_context_set_batch_mode(hms_ctx, mode)
            outs = [np.empty_like(p) for p in loads]
            its = np.zeros(nrhs, np.int32)
            capi.hms_solve_batch(hms_ctx, prs, loads, outs, iters=its)
            res[mode] = (outs, its)
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_AUTO)
        (ol, il), (os_, is_) = res[capi.HMS_BATCH_LOCKSTEP], res[capi.HMS_BATCH_STREAMS]
        assert np.array_equal(il, is_)
        k = 0
        for l, pr, p, a, b in zip(lats, prs, loads, ol, os_):
            assert np.array_equal(a, b), (l.nx, l.ny)
            solo = np.empty_like(p)
            sits = np.zeros(l.nrhs, np.int32)
            capi.hms_solve(hms_ctx, pr, p, solo, iters=sits)
            assert np.array_equal(a, solo) and np.array_equal(il[k:k + l.nrhs], sits)
            k += l.nrhs
    finally:
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_AUTO)
        for pr in prs:
            capi.hms_problem_destroy(pr)


def test_lockstep_refuses_mixed_precisions(hms_ctx):
    from paper_1208_4093_gb300 import capi
    a = capi.hms_problem_create(hms_ctx, 40, 40, 16, 16, precision=0, coarse_factor=4)
    b = capi.hms_problem_create(hms_ctx, 40, 40, 16, 16, precision=1, coarse_factor=4)
    try:
        p = np.zeros((1, 2 * 40 * 40))
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_LOCKSTEP)
        with pytest.raises(capi.HmsError) as e:
            capi.hms_solve_batch(hms_ctx, [a, b], [p, p], [np.empty_like(p), np.empty_like(p)])
        assert e.value.status == capi.HMS_ERR_ARG
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_AUTO)
        capi.hms_solve_batch(hms_ctx, [a, b], [p, p], [np.empty_like(p), np.empty_like(p)])  # streams
        with pytest.raises(capi.HmsError):
            capi.hms_context_set_batch_mode(hms_ctx, 7)
    finally:
        capi.hms_context_set_batch_mode(hms_ctx, capi.HMS_BATCH_AUTO)
        capi.hms_problem_destroy(a)
        capi.hms_problem_destroy(b)
