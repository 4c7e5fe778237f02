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
