"""Pins for the oracle's pruning statistics (Table 1 of Section 3: nodes
visited by the downward pass under neighbor pruning and under distance
pruning), checked against brute force on the tree's structure, closed forms
and limits."""
import numpy as np

import oracle
from paper_1410_0260_gb300 import workloads as wl


def _ranges(N, L):
    """Node ranges of the median-split tree: left child ceil(n/2)."""
    start, size = {1: 0}, {1: N}
    for a in range(1, 1 << L):
        n = size[a]
        start[2 * a], size[2 * a] = start[a], (n + 1) // 2
        start[2 * a + 1], size[2 * a + 1] = start[a] + (n + 1) // 2, n // 2
    return start, size


def _brute(X, m, kappa, rscale, targets):
    perm, L = oracle.askit_tree(X, m)
    N = len(X)
    start, size = _ranges(N, L)
    X64 = X.astype(np.float64)
    nodes = range(1, 2 << L)
    cent = {a: X64[perm[start[a]: start[a] + size[a]]].mean(0) for a in nodes}
    r2 = {a: ((X64[perm[start[a]: start[a] + size[a]]] - cent[a]) ** 2).sum(1).max() for a in nodes}
    leaf = np.empty(N, np.int64)
    for a in range(1 << L, 2 << L):
        leaf[perm[start[a]: start[a] + size[a]]] = a
    ids, _ = oracle.knn_exact(X, kappa)
    out = []
    for i in targets:
        U = set()
        for lf in {leaf[i]} | {leaf[j] for j in ids[i]}:
            while lf >= 1:
                U.add(lf)
                lf >>= 1
        vk = len(U) + sum(1 for a in U if a < (1 << L) for c in (2 * a, 2 * a + 1) if c not in U)

        def vd(a, depth):
            if depth > 0 and ((X64[i] - cent[a]) ** 2).sum() > rscale ** 2 * r2[a]:
                return 1
            if depth == L:
                return 1
            return 1 + vd(2 * a, depth + 1) + vd(2 * a + 1, depth + 1)
        out.append((vk, vd(1, 0)))
    return L, out


def test_prune_stats_match_brute_force():
    for X in (wl.gaussian(700, 3, 1), wl.curve(600, 8, 2), wl.hypersphere(650, 6, 3)):
        L, vk, vd = oracle.prune_stats(X, 16, 12, 1.0)
        tg = [0, 7, 123, len(X) - 1]
        Lb, ref = _brute(X, 16, 12, 1.0, tg)
        assert L == Lb
        for t, (rk, rd) in zip(tg, ref):
            # the centroids differ from numpy's mean only by summation order,
            # which can flip a test at exact ties only
            assert vk[t] == rk, t
            assert abs(vd[t] - rd) <= 2, (t, vd[t], rd)


def test_prune_stats_limits():
    X = wl.gaussian(512, 4, 5)
    L, vk, vd = oracle.prune_stats(X, 16, 511, 1e6)
    total = (2 << L) - 1
    assert (vk == total).all() and (vd == total).all()       # nothing pruned
    L, vk, vd = oracle.prune_stats(X, 16, 1, 0.0)
    assert (vd == 3).all()                                   # every child of the root pruned
    assert (vk >= 1 + 2 * L).all() and (vk <= 1 + 4 * L).all()   # one or two root-to-leaf paths


def test_curve_prunes_better_than_gaussian_in_high_dimension():
    """The trend Table 1 reports: at 32 dimensions neighbor pruning visits far
    fewer nodes on the curve than on the Gaussian, and distance pruning visits
    nearly every node of the Gaussian's tree."""
    N, m, kappa = 4096, 64, 64
    Lg, vkg, vdg = oracle.prune_stats(wl.gaussian(N, 32, 7), m, kappa, 1.0)
    Lc, vkc, vdc = oracle.prune_stats(wl.curve(N, 32, 7), m, kappa, 1.0)
    tot = (2 << Lg) - 1
    assert vkc.mean() < vkg.mean()
    assert vdg.mean() / tot > 0.9
