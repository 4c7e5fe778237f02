"""Relaxation CTA size and copies per matrix: every size gives bitwise the
same iteration, and the autotuned choice (relax_threads = 0) is one of them,
kept per set shape.

The relaxation's row sums are formed by groups of 4 threads whatever the CTA
size, and its P sums over 256 virtual lanes, so 64-, 128- and 256-thread CTAs
must produce identical bits; the autotuner only changes the time."""
import numpy as np
import pytest

from workloads import ea_lognormal, loads

pytestmark = pytest.mark.gpu

# nx, ny, sx, sy, lognormal EA: 32 x 32 sets with ragged edges, and 64-wide sets
SHAPES = [(70, 45, 32, 32, True), (130, 40, 64, 16, False)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: f"{s[0]}x{s[1]}_sets{s[2]}x{s[3]}")
@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
def test_every_cta_size_gives_the_same_bits(hms_ctx, shape, prec):
    from paper_1208_4093_gb300 import capi
    nx, ny, sx, sy, ln = shape
    kw = dict(precision=prec, tol=1e-9, max_iter=3000)
    if ln:
        kw["ea"] = ea_lognormal(nx, ny, 3)
    p = loads(nx, ny, 8).reshape(1, -1)
    r = loads(nx, ny, 9).reshape(-1)
    outs, its, rel = [], [], []
    # two copies per matrix: FP64 and even set widths >= 6 (the ragged 6-wide column included)
    two = prec == 0 and sx % 2 == 0 and (nx - (-(-nx // sx) - 1) * sx) % 2 == 0 and nx - (-(-nx // sx) - 1) * sx >= 6
    variants = [(64, 1), (128, 1), (256, 1), (0, 0)] + ([(64, 2), (128, 2), (256, 2)] if two else [])
    if not two:
        with pytest.raises(capi.HmsError) as e:
            capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, relax_threads=128, relax_copies=2, **kw)
        assert e.value.status == capi.HMS_ERR_ARG
    for nt, nc in variants:
        pr = capi.hms_problem_create(hms_ctx, nx, ny, sx, sy, relax_threads=nt, relax_copies=nc, **kw)
        try:
            got = capi.hms_problem_relax_threads(pr)
            assert got == nt if nt else got in (64, 128, 256)
            gc = capi.hms_problem_relax_copies(pr)
            assert gc == nc if nc else gc in ((1, 2) if two else (1,))
            u = np.empty_like(p)
            it = np.zeros(1, np.int32)
            capi.hms_solve(hms_ctx, pr, p, u, iters=it)
            outs.append(u)
            its.append(int(it[0]))
            d = np.empty(2 * nx * ny)
            P = np.empty(9 * (-(-nx // sx)) * (-(-ny // sy)))
            capi.hms_relax(hms_ctx, pr, r, d, P)
            rel.append((d, P))
        finally:
            capi.hms_problem_destroy(pr)
    for k in range(1, len(variants)):
        assert np.array_equal(outs[k], outs[0])
        assert its[k] == its[0]
        assert np.array_equal(rel[k][0], rel[0][0]) and np.array_equal(rel[k][1], rel[0][1])


def test_autotuned_choice_is_kept_per_set_shape(hms_ctx):
    from paper_1208_4093_gb300 import capi
    a = capi.hms_problem_create(hms_ctx, 96, 64, 32, 32, precision=1)
    b = capi.hms_problem_create(hms_ctx, 160, 96, 32, 32, precision=1)
    try:
        assert capi.hms_problem_relax_threads(a) == capi.hms_problem_relax_threads(b)
        c = capi.hms_problem_clone(hms_ctx, a)
        assert capi.hms_problem_relax_threads(c) == capi.hms_problem_relax_threads(a)
        capi.hms_problem_destroy(c)
    finally:
        capi.hms_problem_destroy(a)
        capi.hms_problem_destroy(b)


@pytest.mark.parametrize("nt", [-1, 32, 100, 512])
def test_bad_cta_size_rejected(hms_ctx, nt):
    from paper_1208_4093_gb300 import capi
    with pytest.raises(capi.HmsError) as e:
        capi.hms_problem_create(hms_ctx, 16, 16, 8, 8, relax_threads=nt)
    assert e.value.status == capi.HMS_ERR_ARG
