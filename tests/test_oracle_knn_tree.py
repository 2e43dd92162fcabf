"""Pins for the oracle's kNN (exact and random-projection trees, Section 2.2)
and for its binary tree (Section 2.2 split rule, Fig. 3).

kNN is checked against brute force with exact integer arithmetic (so ties
by index are exercised), the RP search against exact kNN when one leaf holds
every point, and monotonicity in the number of trees.  The tree is checked
on hand-built cases whose split is known by inspection, on collinear data,
and on leaf sizes for ragged N.
"""
import numpy as np
import pytest

import oracle


def brute_knn_int(Xi, kappa):
    """kNN by exact integer distances, ties broken by index (numpy.lexsort)."""
    N = Xi.shape[0]
    D = ((Xi[:, None, :] - Xi[None, :, :]) ** 2).sum(-1)
    ids = np.zeros((N, kappa), np.int64)
    for i in range(N):
        order = np.lexsort((np.arange(N), D[i]))
        order = order[order != i][:kappa]
        ids[i] = order
    return ids, D


def test_exact_knn_with_ties_matches_brute_force():
    rng = np.random.default_rng(0)
    Xi = rng.integers(0, 4, size=(300, 3))          # many duplicate points and equal distances
    ids, dd = oracle.knn_exact(Xi.astype(np.float32), 10)
    ref, D = brute_knn_int(Xi, 10)
    assert np.array_equal(ids, ref)
    assert np.array_equal(dd, np.take_along_axis(D, ref, 1).astype(np.float64))


def test_exact_knn_out_of_sample_queries():
    rng = np.random.default_rng(1)
    Xi = rng.integers(-5, 5, size=(200, 4))
    Yi = rng.integers(-5, 5, size=(30, 4))
    ids, _ = oracle.knn_exact(Xi.astype(np.float32), 7, Y=Yi.astype(np.float32))
    D = ((Yi[:, None, :] - Xi[None, :, :]) ** 2).sum(-1)
    for q in range(30):
        assert np.array_equal(ids[q], np.lexsort((np.arange(200), D[q]))[:7])   # no self-exclusion


def test_rp_knn_single_leaf_is_exact():
    rng = np.random.default_rng(2)
    X = rng.standard_normal((180, 6)).astype(np.float32)
    ids_rp, d_rp = oracle.knn_rp(X, 12, 2, 4096, 99)
    ids_ex, d_ex = oracle.knn_exact(X, 12)
    assert np.array_equal(ids_rp, ids_ex) and np.array_equal(d_rp, d_ex)


def test_rp_knn_valid_and_monotone_in_trees():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((2000, 5)).astype(np.float32)
    k = 8
    prev = None
    ex, dex = oracle.knn_exact(X, k)
    for T in (1, 2, 4, 8):
        ids, dd = oracle.knn_rp(X, k, T, 64, 5)
        # entries valid: not self, distinct, true distances, sorted by (D, j)
        assert (ids != np.arange(2000)[:, None]).all()
        assert all(len(set(r)) == k for r in ids)
        Dtrue = ((X[:, None, :].astype(np.float64) - X[ids].astype(np.float64)) ** 2).sum(-1)
        assert np.allclose(dd, Dtrue, rtol=1e-12, atol=0)
        assert (np.diff(dd, axis=1) >= 0).all()
        # never better than exact, never worse with more trees (the T trees are a prefix of T+1)
        assert (dd >= dex - 0).all()
        if prev is not None:
            assert (dd <= prev).all()
        prev = dd
    hit = np.mean([len(set(a) & set(b)) / k for a, b in zip(ids, ex)])
    assert hit > 0.6


def test_tree_depth_rule():
    assert oracle.tree_depth(4096, 128) == 5
    assert oracle.tree_depth(100, 8) == 4        # ceil(100/16) = 7 <= 8, ceil(100/8) = 13 > 8
    assert oracle.tree_depth(128, 128) == 0


def test_tree_hand_built_split_and_farthest_tie():
    # center (5.5, 0); points 0 and 3 tie as farthest -> smallest id (0) is x_l;
    # x_r = point 3; projections 0, 110, 11, 121 -> left {0, 2}, right {1, 3}
    X = np.array([[0, 0], [10, 0], [1, 0], [11, 0]], np.float32)
    perm, L = oracle.askit_tree(X, 2)
    assert L == 1 and list(perm) == [0, 2, 1, 3]


def test_tree_collinear_points_are_sorted_intervals():
    rng = np.random.default_rng(4)
    N, m = 256, 8
    t = rng.permutation(N).astype(np.float32)          # distinct positions, random order
    X = np.stack([t, 2 * t, -t], 1).astype(np.float32)
    perm, L = oracle.askit_tree(X, m)
    assert L == 5
    leaves = perm.reshape(-1, m)
    for leaf in leaves:
        assert list(leaf) == sorted(leaf)                  # ascending id inside a leaf
        v = np.sort(t[leaf])
        assert v[-1] - v[0] == m - 1                        # a contiguous run of positions
    # left child holds the half nearer the extreme that is farthest from the mean
    dist = np.abs(t.astype(np.float64) - t.astype(np.float64).mean())
    x_l = int(np.flatnonzero(dist == dist.max()).min())       # ties: smallest id
    assert x_l in set(perm[: N // 2])


def test_tree_ragged_leaf_sizes_and_permutation():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((100, 3)).astype(np.float32)
    perm, L = oracle.askit_tree(X, 8)
    assert sorted(perm) == list(range(100))
    sizes = []

    def rec(n, depth):
        if depth == L:
            sizes.append(n)
            return
        rec((n + 1) // 2, depth + 1)
        rec(n // 2, depth + 1)
    rec(100, 0)
    assert sum(sizes) == 100 and max(sizes) <= 8 and min(sizes) >= 1
    off = 0
    for s in sizes:
        leaf = perm[off: off + s]
        assert list(leaf) == sorted(leaf)
        off += s


def test_rp_split_replayed_on_numpy_philox():
    """One RP split (rp_leaf = N/2) replayed from the definition: Rademacher
    direction bits from numpy's Philox keyed (seed, iteration + 1), counter
    (node, word/4), projection order (p, j), left = first ceil(n/2); then
    exhaustive kNN inside each half.  d = 70 spans two 64-bit words."""
    rng = np.random.default_rng(9)
    N, d, k, seed = 300, 70, 5, 1234
    X = rng.standard_normal((N, d)).astype(np.float32)
    ids, dd = oracle.knn_rp(X, k, 1, N // 2, seed)
    words = np.random.Philox(key=seed + (1 << 64), counter=1 - 1).random_raw(4)   # node 1, block 0
    v = np.array([-1.0 if (int(words[kk >> 6]) >> (kk & 63)) & 1 else 1.0 for kk in range(d)])
    p = np.zeros(N)
    for kk in range(d):                    # ascending-k sum, as defined
        p = p + v[kk] * X[:, kk].astype(np.float64)
    order = np.lexsort((np.arange(N), p))
    halves = [np.sort(order[: (N + 1) // 2]), np.sort(order[(N + 1) // 2:])]
    for hv in halves:
        sub = X[hv]
        sid, _ = oracle.knn_exact(sub, k)
        assert np.array_equal(ids[hv], hv[sid])
