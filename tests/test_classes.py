"""Classes of identical sets (class_factors = 1; reading R20) against the
oracle's matrices, on the host: hms_set_classes needs no device.

With a uniform bar stiffness the library puts two sets in one class (one
factor of k^Inner, Eq. 12, shared by all its sets) when they agree in width,
height, parity of the first row, the lattice edges they touch and their
constrained DOFs.  The oracle assembles K bar by bar from node coordinates and
takes each set's k^Inner as the principal submatrix of K on the set's free
DOFs (Eq. 11).  The library's classes must be exactly the groups of sets whose
(k^Inner, constrained DOFs) are the same: every class holds only equal
matrices, and sets of different classes differ.
"""
import numpy as np
import pytest

from oracle import truss


def roller_left(nx, ny):
    f = np.zeros((ny, nx, 2), np.uint8)
    f[0] = 1
    f[:, 0, 0] = 1
    return f


def pinned_spots(nx, ny):
    f = np.zeros((ny, nx, 2), np.uint8)
    f[0] = 1
    f[ny // 2, nx // 3] = 1
    f[ny - 1, nx - 1, 1] = 1
    return f


# nx, ny, sx, sy, supports: 3 x 3 sets with a ragged last row and column (the
# set shapes of the 1e9-DOF lattice, scaled down); odd set height (the first
# row's parity alternates); small sets; a roller edge; scattered supports
CASES = [
    (21, 21, 8, 8, None),
    (26, 23, 8, 7, None),
    (20, 18, 5, 6, None),
    (24, 20, 6, 5, roller_left),
    (24, 24, 6, 6, pinned_spots),
]


def local(K, free, nx, ny, sx, sy, I):
    mx = -(-nx // sx)
    i0, j0 = (I % mx) * sx, (I // mx) * sy
    w, h = min(sx, nx - i0), min(sy, ny - j0)
    idx = np.array([2 * ((j0 + jl) * nx + i0 + il) + d for jl in range(h) for il in range(w) for d in range(2)])
    fl = free[idx]
    k = K[idx][:, idx].toarray()[np.ix_(fl, fl)]
    return (w, h), fl, k


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}_{c[2]}x{c[3]}" + ("" if c[4] is None else "_" + c[4].__name__)
                                             for c in CASES])
def test_classes_are_the_groups_of_equal_local_matrices(case):
    from paper_1208_4093_gb300 import capi
    nx, ny, sx, sy, fb = case
    fixed = fb(nx, ny) if fb else None
    classes, n = capi.hms_set_classes(nx, ny, sx, sy, fixed=fixed)
    K = truss.assemble_K(nx, ny).tocsr()
    free = truss.free_mask(nx, ny, fixed)
    M = len(classes)
    mats = [local(K, free, nx, ny, sx, sy, I) for I in range(M)]

    def same(a, b):
        (sa, fa, ka), (sb, fb_, kb) = mats[a], mats[b]
        if sa != sb or not np.array_equal(fa, fb_):
            return False
        return np.allclose(ka, kb, rtol=0.0, atol=1e-12 * max(1.0, np.abs(ka).max()))

    # classes numbered by first appearance in set order
    assert classes[0] == 0 and n == classes.max() + 1
    assert all(classes[I] <= classes[:I].max(initial=-1) + 1 for I in range(M))
    reps = [int(np.flatnonzero(classes == c)[0]) for c in range(n)]
    for I in range(M):
        assert same(I, reps[classes[I]]), (I, int(classes[I]))
    for a in range(n):
        for b in range(a + 1, n):
            assert not same(reps[a], reps[b]), (a, b)


def test_class_counts():
    from paper_1208_4093_gb300 import capi
    # the 1e9-DOF lattice: 350 x 350 sets of 64 x 64, the last row and column
    # 25 wide, bottom row clamped: first / inner / last set column times
    # first / inner / last set row (the rows all start on even lattice rows)
    classes, n = capi.hms_set_classes(22361, 22361, 64, 64)
    assert n == 9 and len(classes) == 350 * 350
    assert np.bincount(classes).tolist() == [1, 348, 1, 348, 348 * 348, 348, 1, 348, 1]
    with pytest.raises(capi.HmsError):  # bad arguments
        capi.hms_set_classes(1, 64, 16, 16)
