"""Serving: requests of different sizes admitted under an HBM budget and
advanced together (continuous batching) give the same result as solo solves,
and every served load vector matches the oracle's direct solve.

Every request runs its own problem, whose kernels are deterministic and share
no buffers with the others, so each result in the mix must equal its solo
hms_solve bit for bit; the byte estimate used for admission must match what
problem creation allocates.
"""
import numpy as np
import pytest

from workloads import ea_lognormal, loads

pytestmark = pytest.mark.gpu

# nx, ny, sx, sy, lognormal EA, precision (0 FP64, 1 mixed), nrhs
REQS = [
    (48, 40, 16, 16, True, 1, 2),
    (33, 21, 16, 8, False, 0, 1),
    (64, 24, 32, 12, True, 1, 3),
    (20, 52, 10, 13, True, 0, 2),
    (70, 35, 32, 32, False, 1, 1),
    (40, 40, 20, 20, True, 1, 2),
    # 48 x 2 sets: wider than any band factor's window, so the upper level is
    # factored by nested dissection
    (1536, 40, 32, 20, True, 1, 2),
]


def req_args(k, r):
    nx, ny, sx, sy, ln, prec, nrhs = r
    kw = dict(precision=prec, tol=1e-10, max_iter=3000)
    if ln:
        kw["ea"] = ea_lognormal(nx, ny, 50 + k)
    p = np.stack([loads(nx, ny, 60 + k, q).reshape(-1) for q in range(nrhs)])
    return nx, ny, sx, sy, kw, p


def b_size_max():
    # pad4 of the entry count of a B block with nb = 160, the widest relaxation
    # region row (80 nodes; rows r hold columns max(0, r-3)..159)
    nb = 160
    n = sum(nb - max(0, r - 3) for r in range(nb))
    return (n + 3) // 4 * 4


def test_estimate_equals_allocation_plus_setup_scratch(hms_ctx):
    import torch
    from paper_1208_4093_gb300 import capi
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for k, r in enumerate(REQS):
        nx, ny, sx, sy, kw, _ = req_args(k, r)
        est = capi.hms_problem_estimate_bytes(hms_ctx, nx, ny, sx, sy, **kw)
        pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, **kw)
        try:
            got = capi.hms_problem_device_bytes(pr)
        finally:
            capi.hms_problem_destroy(pr)
        m = -(-nx // sx) * -(-ny // sy)
        assert est - got == min(m, nsm) * b_size_max() * 8, (r, est, got)
    assert capi.hms_problem_estimate_bytes(hms_ctx, 8, 8, 65, 4) == 0


def test_serving_matches_solo(hms_ctx):
    from oracle import direct, truss
    from paper_1208_4093_gb300 import capi
    srv = capi.hms_server_create(hms_ctx, 64 << 30, max_active=64)
    ids = {}
    try:
        # first wave, two rounds, then the second wave joins the running ones
        for k in range(3):
            nx, ny, sx, sy, kw, p = req_args(k, REQS[k])
            ids[capi.hms_server_submit(hms_ctx, srv, nx, ny, sx, sy, p, **kw)] = k
        finished = []
        for _ in range(2):
            finished += capi.hms_server_step(hms_ctx, srv)[0]
        for k in range(3, len(REQS)):
            nx, ny, sx, sy, kw, p = req_args(k, REQS[k])
            ids[capi.hms_server_submit(hms_ctx, srv, nx, ny, sx, sy, p, **kw)] = k
        for _ in range(5000):
            done, na, nq, used = capi.hms_server_step(hms_ctx, srv)
            finished += done
            if na == 0 and nq == 0:
                break
        assert sorted(finished) == sorted(ids)
        for rid, k in ids.items():
            nx, ny, sx, sy, kw, p = req_args(k, REQS[k])
            u = np.empty_like(p)
            its = np.zeros(p.shape[0], np.int32)
            assert capi.hms_server_take(hms_ctx, srv, rid, u, its) == capi.HMS_OK
            pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, **kw)
            try:
                solo = np.empty_like(p)
                sits = np.zeros(p.shape[0], np.int32)
                capi.hms_solve(hms_ctx, pr, p, solo, iters=sits)
            finally:
                capi.hms_problem_destroy(pr)
            assert np.array_equal(u, solo), REQS[k]
            assert np.array_equal(its, sits)
            # and every served load vector against the direct solve (O1):
            # 1e-9 for the FP64 path, 1e-8 for the mixed one
            tr = truss.Truss(nx, ny, kw.get("ea"))
            bar = 1e-9 if kw["precision"] == capi.HMS_FP64 else 1e-8
            for q in range(p.shape[0]):
                us = direct.sparse_solve(tr, tr.free * p[q])
                assert np.linalg.norm(u[q] - us) <= bar * np.linalg.norm(us), (REQS[k], q)
    finally:
        capi.hms_server_destroy(srv)


def test_budget_admission_and_rejections(hms_ctx):
    from paper_1208_4093_gb300 import capi
    sizes = []
    for k, r in enumerate(REQS):
        nx, ny, sx, sy, kw, _ = req_args(k, r)
        sizes.append(capi.hms_problem_estimate_bytes(hms_ctx, nx, ny, sx, sy, **kw))
    # a request holds its shared setup plus one instance per load vector (<= 3 here)
    budget = 3 * max(sizes)
    srv = capi.hms_server_create(hms_ctx, budget, max_active=8)
    try:
        nx, ny, sx, sy, kw, p = req_args(0, REQS[0])
        with pytest.raises(capi.HmsError) as e:
            capi.hms_server_submit(hms_ctx, srv, 64, 64, 65, 8, np.zeros((1, 2 * 64 * 64)))
        assert e.value.status == capi.HMS_ERR_ARG
        big = capi.hms_server_create(hms_ctx, 1 << 20, max_active=8)
        try:
            with pytest.raises(capi.HmsError) as e:
                capi.hms_server_submit(hms_ctx, big, nx, ny, sx, sy, p, **kw)
            assert e.value.status == capi.HMS_ERR_OOM
        finally:
            capi.hms_server_destroy(big)
        ids = []
        for k, r in enumerate(REQS):
            nx, ny, sx, sy, kw, p = req_args(k, r)
            ids.append(capi.hms_server_submit(hms_ctx, srv, nx, ny, sx, sy, p, **kw))
        done = []
        for _ in range(10000):
            d, na, nq, used = capi.hms_server_step(hms_ctx, srv)
            assert used <= budget
            done += d
            if na == 0 and nq == 0:
                break
        assert sorted(done) == sorted(ids)
        for rid in ids:
            assert capi.hms_server_take(hms_ctx, srv, rid) == capi.HMS_OK
    finally:
        capi.hms_server_destroy(srv)


def test_clone_shares_setup_and_outlives_its_source(hms_ctx):
    from paper_1208_4093_gb300 import capi
    nx, ny, sx, sy, kw, p = req_args(0, REQS[0])
    pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, **kw)
    cl = capi.hms_problem_clone(hms_ctx, pr)
    try:
        assert capi.hms_problem_device_bytes(cl) < capi.hms_problem_device_bytes(pr)
        a, b = np.empty_like(p), np.empty_like(p)
        capi.hms_solve(hms_ctx, pr, p, a)
        capi.hms_solve(hms_ctx, cl, p, b)
        assert np.array_equal(a, b)
        # both at once, one load vector each
        c0, c1 = np.empty_like(p[:1]), np.empty_like(p[1:2])
        capi.hms_solve_batch(hms_ctx, [pr, cl], [p[:1], p[1:2]], [c0, c1])
        assert np.array_equal(c0, a[:1]) and np.array_equal(c1, a[1:2])
        capi.hms_problem_destroy(pr)
        pr = None
        d = np.empty_like(p)
        capi.hms_solve(hms_ctx, cl, p, d)  # the shared factors live on with the clone
        assert np.array_equal(d, a)
    finally:
        if pr is not None:
            capi.hms_problem_destroy(pr)
        capi.hms_problem_destroy(cl)
