"""The upper level's nested-dissection plan (host logic, no GPU): hms_nd_plan.

K_aa (Eq. 6) couples a set's modes only to those of its eight neighbours in
the set grid, so a tree of separators (set rows or columns cutting boxes of
sets in two) orders Eq. 8 for a multifrontal Cholesky.  These tests check the
plan the library factors by:
* it is an elimination tree: every set eliminated by exactly one node,
  children before parents, one root;
* each node's boundary B is exactly the sets outside its subtree that couple
  to a set inside it, and all of them lie on its ancestors' separators; its
  children's boundaries fall inside its own front, and two sibling subtrees
  never couple;
* a multifrontal factorisation driven by the plan (dense fronts, extend-add of
  the children's update matrices, partial Cholesky of each node's own sets)
  solves a random SPD system with K_aa's block pattern as a dense solve does.
"""
import numpy as np
import pytest


def neighbours(I, mx, my):
    x, y = I % mx, I // mx
    out = []
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if (dx or dy) and 0 <= x + dx < mx and 0 <= y + dy < my:
                out.append((y + dy) * mx + x + dx)
    return out


def plan(mx, my):
    from paper_1208_4093_gb300 import capi
    nodes = capi.hms_nd_plan(mx, my)
    sub = []
    for n in nodes:
        s = set(n["S"])
        for c in n["children"]:
            s |= sub[c]
        sub.append(s)
    parent = {}
    for k, n in enumerate(nodes):
        for c in n["children"]:
            parent[c] = k
    return nodes, sub, parent


@pytest.mark.parametrize("mx,my", [(1, 1), (2, 2), (3, 1), (1, 5), (5, 4), (7, 7), (16, 16), (22, 9), (3, 17)])
def test_nd_plan_is_an_elimination_tree(mx, my):
    nodes, sub, parent = plan(mx, my)
    M = mx * my
    assert sorted(s for n in nodes for s in n["S"]) == list(range(M))
    for k, n in enumerate(nodes):
        assert all(c < k for c in n["children"])
        assert len(set(n["S"])) == len(n["S"]) and len(set(n["B"])) == len(n["B"])
    assert [k for k in range(len(nodes)) if k not in parent] == [len(nodes) - 1]
    assert sum(len(n["children"]) for n in nodes) == len(parent)
    for k, n in enumerate(nodes):
        ring = {J for I in sub[k] for J in neighbours(I, mx, my)} - sub[k]
        assert set(n["B"]) == ring, k
        anc, a = set(), k
        while a in parent:
            a = parent[a]
            anc |= set(nodes[a]["S"])
        assert set(n["B"]) <= anc, k
        front = set(n["S"]) | set(n["B"])
        for c in n["children"]:
            assert set(nodes[c]["B"]) <= front, (k, c)
        if len(n["children"]) == 2:
            a, b = (sub[c] for c in n["children"])
            assert not any(J in b for I in a for J in neighbours(I, mx, my)), k


def multifrontal_solve(A, rhs, nodes, q):
    """Solve A x = rhs with the plan: per node a dense front over S then B."""
    def idx(sets):
        return np.array([s * q + m for s in sets for m in range(q)], dtype=int)
    upd, fac = {}, {}
    for k, n in enumerate(nodes):
        S, B = n["S"], n["B"]
        f = idx(S + B)
        ns = q * len(S)
        F = np.zeros((len(f), len(f)))
        # the original entries of this node's own rows (and their mirror)
        F[:ns, :] = A[np.ix_(f[:ns], f)]
        F[ns:, :ns] = A[np.ix_(f[ns:], f[:ns])]
        # extend-add of the children's update matrices (over their boundaries)
        pos = {s: t for t, s in enumerate(S + B)}
        for c in n["children"]:
            cb = nodes[c]["B"]
            where = np.array([pos[s] * q + m for s in cb for m in range(q)], dtype=int)
            F[np.ix_(where, where)] += upd.pop(c)
        L11 = np.linalg.cholesky(F[:ns, :ns])
        L21 = np.linalg.solve(L11, F[:ns, ns:]).T
        upd[k] = F[ns:, ns:] - L21 @ L21.T
        fac[k] = (f, ns, L11, L21)
    y = rhs.copy()
    for k in range(len(nodes)):                 # forward, children first
        f, ns, L11, L21 = fac[k]
        ys = np.linalg.solve(L11, y[f[:ns]])
        y[f[:ns]] = ys
        y[f[ns:]] -= L21 @ ys
    x = y.copy()
    for k in reversed(range(len(nodes))):       # backward, root first
        f, ns, L11, L21 = fac[k]
        x[f[:ns]] = np.linalg.solve(L11.T, y[f[:ns]] - L21.T @ x[f[ns:]])
    return x


@pytest.mark.parametrize("mx,my,q", [(5, 4, 2), (7, 7, 1), (9, 6, 3), (4, 11, 9)])
def test_nd_plan_factor_solves_a_set_grid_system(mx, my, q):
    nodes, _, _ = plan(mx, my)
    rng = np.random.default_rng(mx * 100 + my)
    M = mx * my
    n = M * q
    A = np.zeros((n, n))
    for I in range(M):
        for J in neighbours(I, mx, my) + [I]:
            if J < I:
                continue
            blk = rng.standard_normal((q, q))
            if J == I:
                blk = blk + blk.T
            A[I * q:(I + 1) * q, J * q:(J + 1) * q] = blk
            A[J * q:(J + 1) * q, I * q:(I + 1) * q] = blk.T
    A += np.diag(np.abs(A).sum(axis=1) + 1.0)  # symmetric, strictly diagonally dominant: SPD
    rhs = rng.standard_normal(n)
    x = multifrontal_solve(A, rhs, nodes, q)
    want = np.linalg.solve(A, rhs)
    assert np.linalg.norm(x - want) <= 1e-12 * np.linalg.norm(want)


def test_planted_plan_mistakes_are_caught():
    """A plan with one boundary set missing from a leaf's front no longer
    solves the system: the multifrontal check is not vacuous."""
    import copy
    mx, my, q = 7, 5, 2
    nodes, _, _ = plan(mx, my)
    rng = np.random.default_rng(1)
    M = mx * my
    A = np.zeros((M * q, M * q))
    for I in range(M):
        for J in neighbours(I, mx, my) + [I]:
            if J >= I:
                blk = rng.standard_normal((q, q))
                A[I * q:(I + 1) * q, J * q:(J + 1) * q] = blk + (blk.T if J == I else 0)
                A[J * q:(J + 1) * q, I * q:(I + 1) * q] = A[I * q:(I + 1) * q, J * q:(J + 1) * q].T
    A += np.diag(np.abs(A).sum(axis=1) + 1.0)
    rhs = rng.standard_normal(M * q)
    want = np.linalg.solve(A, rhs)
    # a leaf's boundary loses a set (its coupling to that set is dropped)
    bad = copy.deepcopy(nodes)
    k = next(i for i, n in enumerate(bad) if not n["children"] and len(n["B"]) > 1)
    bad[k]["B"] = bad[k]["B"][1:]
    x = multifrontal_solve(A, rhs, bad, q)
    assert np.linalg.norm(x - want) > 1e-6 * np.linalg.norm(want)
