"""The balanced relaxation schedule (host logic, no GPU): hms_relax_schedule.

The library cuts the sets' substitution steps into one equal share per
persistent CTA by McNaughton's wrap-around rule: a set cut between CTAs g-1
and g has its head run first by CTA g-1 and its tail run last by CTA g.  These
tests check, with their own cost model (one FMA per factor entry of each op's
matrix, the factor layout of the block-bidiagonal Cholesky factor of Eq. 12's
k^Inner), that
* every set's ops are covered exactly once and in order, cut only where the
  substitution's state is in device memory (after a Linv_j product of the
  forward pass, or a Linv_j^T product of the backward pass);
* each CTA runs at most one head (first) and one tail (last);
* the busiest CTA carries little more than the mean share, where one CTA per
  set in waves of the CTA count carries up to twice as much;
* replayed in time at one FMA per unit, no tail starts before its head ends
  (so in a balanced run no CTA waits for another).
"""
import numpy as np
import pytest


def op_entries(nb, h):
    """FMA count of each op of a set with h rows of nb DOFs: forward ops
    Linv_0, B_1, Linv_1, ..., then the same matrices in reverse."""
    linv = nb * (nb + 1) // 2
    b = sum(nb - max(0, r - 3) for r in range(nb))
    nmat = 2 * h - 1
    fwd = [linv if k % 2 == 0 else b for k in range(nmat)]
    return fwd + fwd[::-1]


def set_shape(nx, ny, sx, sy, I):
    mx = -(-nx // sx)
    i0, j0 = (I % mx) * sx, (I // mx) * sy
    return 2 * min(sx, nx - i0), min(sy, ny - j0)


def check(nx, ny, sx, sy, ctas):
    from paper_1208_4093_gb300 import capi
    res = capi.hms_relax_schedule(nx, ny, sx, sy, ctas)
    assert res is not None
    segs, cta = res
    M = (-(-nx // sx)) * (-(-ny // sy))
    assert cta[0] == 0 and cta[-1] == len(segs) and np.all(np.diff(cta) >= 1)
    costs = {I: np.cumsum([0] + op_entries(*set_shape(nx, ny, sx, sy, I))) for I in range(M)}
    parts = {}
    finish, start = {}, {}
    loads = []
    for g in range(ctas):
        t = 0.0
        for k in range(cta[g], cta[g + 1]):
            I, o0, o1 = (int(x) for x in segs[k])
            c = costs[I]
            nops = len(c) - 1
            nmat = nops // 2
            assert 0 <= o0 < o1 <= nops
            for cut in (o0, o1):
                assert cut in (0, nops) or (cut % 2 == 1 and cut <= nmat) or (cut % 2 == 0 and cut > nmat), (I, cut)
            if o1 < nops:
                assert k == cta[g], "a head runs first"
                finish[I] = (g, t + c[o1] - c[o0])
            if o0 > 0:
                assert k == cta[g + 1] - 1, "a tail runs last"
                start[I] = (g, t)
            parts.setdefault(I, []).append((o0, o1))
            t += c[o1] - c[o0]
        loads.append(t)
    # every set exactly once, in order
    assert sorted(parts) == list(range(M))
    for I, p in parts.items():
        p = sorted(p)
        assert p[0][0] == 0 and p[-1][1] == len(costs[I]) - 1
        assert all(a[1] == b[0] for a, b in zip(p, p[1:])) and len(p) <= 2
    # a cut set: head on CTA g-1, tail on CTA g, the tail starting after the head ends
    assert sorted(finish) == sorted(start)
    for I in finish:
        (gh, th), (gt, tt) = finish[I], start[I]
        assert gt == gh + 1
        assert tt >= th, (I, th, tt)
    mean = sum(loads) / ctas
    waves = [0.0] * ctas
    for I in range(M):
        waves[I % ctas] += costs[I][-1]
    return max(loads) / mean, max(waves) / mean, len(finish)


@pytest.mark.parametrize("nx,ny,sx,sy,bound", [
    (1024, 1024, 64, 64, 1.02),   # the 1024^2 workload: 256 sets, 1.68 per CTA
    (120, 112, 8, 8, 1.08),       # 210 sets (small ops: the library also weighs each op's fixed cost)
    (118, 110, 8, 8, 1.08),       # ragged last row and column of sets
    (2048, 256, 32, 32, 1.01),
    (70, 300, 5, 7, 1.02),
])
def test_schedule_covers_balances_and_never_waits(nx, ny, sx, sy, bound):
    busiest, waves, cut = check(nx, ny, sx, sy, 152)
    assert busiest <= bound, busiest
    assert cut > 0
    assert busiest <= waves + 1e-12


def test_schedule_on_the_workload_beats_waves():
    busiest, waves, cut = check(1024, 1024, 64, 64, 152)
    # one CTA per set: 104 SMs run two sets, 48 one (the mean is 256 / 152)
    assert waves == pytest.approx(2 * 152 / 256, rel=1e-12)
    assert busiest < 1.02


def test_schedule_does_not_apply():
    from paper_1208_4093_gb300 import capi
    assert capi.hms_relax_schedule(64, 64, 16, 16, 152) is None     # 16 sets, fewer than the CTAs
    assert capi.hms_relax_schedule(1024, 1024, 64, 64, 256) is None  # one set per CTA
    with pytest.raises(capi.HmsError):
        capi.hms_relax_schedule(1, 64, 16, 16, 152)
    with pytest.raises(capi.HmsError):
        capi.hms_relax_schedule(64, 64, 65, 16, 152)


def test_schedule_handoff_reproduces_the_substitution():
    """Run every set's block substitution (Eq. 12's local solve, k^Inner = L L^T
    with L block bidiagonal by lattice rows) op by op in the plan's segments, a
    cut set's tail starting only from what the head left in device memory: y_j
    after a forward Linv_j product (o0 <= 2h - 1), x_j (the set's delta row j)
    after a backward Linv_j^T product.  Every set must get k^Inner^-1 r_I."""
    import numpy as np
    from oracle import truss
    from paper_1208_4093_gb300 import capi
    nx, ny, sx, sy, ctas = 20, 16, 4, 4, 6
    segs, cta = capi.hms_relax_schedule(nx, ny, sx, sy, ctas)
    K = truss.assemble_K(nx, ny).toarray()
    free = truss.free_mask(nx, ny)
    mx = -(-nx // sx)
    rng = np.random.default_rng(3)
    r = free * rng.standard_normal(2 * nx * ny)
    state = {}

    def setup(I):
        i0, j0 = (I % mx) * sx, (I // mx) * sy
        w, h = min(sx, nx - i0), min(sy, ny - j0)
        nb = 2 * w
        idx = np.array([2 * ((j0 + jl) * nx + i0 + il) + d for jl in range(h) for il in range(w) for d in range(2)])
        k = K[np.ix_(idx, idx)].copy()
        fx = ~free[idx]
        k[fx, :] = 0.0
        k[:, fx] = 0.0
        k[fx, fx] = 1.0
        L = np.linalg.cholesky(k)
        blk = lambda a, b: L[a * nb:(a + 1) * nb, b * nb:(b + 1) * nb]
        return dict(h=h, nb=nb, idx=idx, k=k, Linv=[np.linalg.inv(blk(j, j)) for j in range(h)],
                    B=[None] + [blk(j, j - 1) for j in range(1, h)], rr=r[idx].reshape(h, nb),
                    y=np.zeros((h, nb)), x=np.zeros((h, nb)))

    def run(I, o0, o1):
        s = state.setdefault(I, setup(I))
        h, nmat = s["h"], 2 * s["h"] - 1
        # the state a segment starts from: only what device memory holds
        if o0 == 0:
            z = s["rr"][0].copy()
        elif o0 <= nmat:
            ycur = s["y"][(o0 - 1) // 2].copy()
        else:
            xbuf = s["x"][(2 * nmat - o0) // 2].copy()
        for o in range(o0, o1):
            k = o if o < nmat else 2 * nmat - 1 - o
            if o < nmat and k % 2 == 1:          # z = r_j - B_j y_{j-1}
                j = (k + 1) // 2
                z = s["rr"][j] - s["B"][j] @ ycur
            elif o < nmat:                        # y_j = Linv_j z
                j = k // 2
                ycur = s["Linv"][j] @ z
                s["y"][j] = ycur
            elif k % 2 == 0:                      # x_j = Linv_j^T w
                j = k // 2
                wv = ycur if j == h - 1 else wbuf
                xbuf = s["Linv"][j].T @ wv
                s["x"][j] = xbuf
            else:                                 # w = y_{j-1} - B_j^T x_j
                j = (k + 1) // 2
                wbuf = s["y"][j - 1] - s["B"][j].T @ xbuf
        # (locals of a segment end with it: the next segment of the same set
        # is a tail on another CTA)

    heads = [tuple(int(v) for v in segs[cta[g]]) for g in range(ctas)]
    done = set()
    for I, o0, o1 in heads:          # heads wait for nothing
        if o1 < 2 * (2 * state.setdefault(I, setup(I))["h"] - 1):
            run(I, o0, o1)
            done.add((I, o0))
    for g in range(ctas):            # then each CTA's whole sets and tail, in its order
        for k in range(cta[g], cta[g + 1]):
            I, o0, o1 = (int(v) for v in segs[k])
            if (I, o0) not in done:
                run(I, o0, o1)
    for I, s in state.items():
        want = np.linalg.solve(s["k"], r[s["idx"]])
        assert np.allclose(s["x"].reshape(-1), want, rtol=0, atol=1e-10 * np.abs(want).max()), I
    assert len(state) == (-(-nx // sx)) * (-(-ny // sy))
