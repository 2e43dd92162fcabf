"""Pins for the oracle's Evaluate (Algorithm 4 with the pruning rule of
eq. (2.5)): the cases in which ASKIT reduces to the direct sum of eq. (1.1),
the closed-form count of directly evaluated leaves, the bounds of Section 3
on visited nodes, an independent list-form evaluation, linearity in w, and
the trend of the error with the skeleton size (Table 4)."""
import numpy as np
import pytest

import oracle
from paper_1410_0260_gb300 import workloads as wl


def _data(N=512, d=4, seed=0):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((N, d)) + rng.integers(0, 4, (N, 1)) * 3.0).astype(np.float32)
    W = rng.standard_normal((N, 1))
    return X, W


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_full_rank_skeletons_reproduce_direct_sum():
    X, W = _data()
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=8, s_max=100000, id_tol=0.0, h=1.0))
    T.set_weights(W)
    U = T.evaluate()
    assert rel(U, oracle.direct(X, W, 1.0, 0.5, targets=np.arange(len(X)))) < 1e-13


def test_pruning_off_is_direct_sum():
    X, W = _data(seed=1)
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=8, s_max=4, id_tol=0.0, h=1.0, prune=0))
    T.set_weights(W)
    assert rel(T.evaluate(), oracle.direct(X, W, 1.0, 0.5, targets=np.arange(len(X)))) < 1e-13


def test_all_neighbors_means_nothing_prunes():
    X, W = _data(N=128, seed=2)
    T = oracle.Tree(X, oracle.Config(leaf_size=16, kappa=127, s_max=4, id_tol=0.0, h=1.0))
    T.set_weights(W)
    U, near, far = T.evaluate(counts=True)
    assert (far == 0).all() and (near == 8).all()
    assert rel(U, oracle.direct(X, W, 1.0, 0.5, targets=np.arange(128))) < 1e-13


def test_single_leaf_is_direct_sum():
    X, W = _data(N=100, seed=3)
    T = oracle.Tree(X, oracle.Config(leaf_size=128, kappa=5, s_max=4, h=1.0))
    assert T.L == 0
    T.set_weights(W)
    assert rel(T.evaluate(), oracle.direct(X, W, 1.0, 0.5, targets=np.arange(100))) < 1e-13


def _lists(T, i):
    """Near leaves and far nodes of target i from the definition of U_i."""
    ids, _ = T.knn()
    perm = T.perm()
    c = T.counts()
    L = T.L
    leafof = np.zeros(T.N, np.int64)
    for a in range(1 << L, 2 << L):
        leafof[perm[c["start"][a]: c["start"][a] + c["size"][a]]] = a
    near = sorted({int(leafof[j]) for j in [i] + list(ids[i])})
    U = set()
    for lf in near:
        a = lf
        while a >= 1:
            U.add(a)
            a //= 2
    far = sorted({b ^ 1 for b in U if b > 1 and (b ^ 1) not in U})
    return near, far, leafof


def test_visited_counts_closed_form_and_bounds():
    X, W = _data(N=1024, seed=4)
    cfg = oracle.Config(leaf_size=32, kappa=10, s_max=8, id_tol=1e-3, h=1.0)
    T = oracle.Tree(X, cfg)
    T.set_weights(W)
    _, near, far = T.evaluate(counts=True)
    for i in range(0, 1024, 37):
        nl, fl, _ = _lists(T, i)
        assert near[i] == len(nl) and far[i] == len(fl)
    assert (near <= cfg.kappa + 1).all()
    assert (far <= (cfg.kappa + 1) * T.L).all()


def test_list_form_equals_recursive_form():
    H2 = float(np.float32(1.2)) ** 2     # bandwidths are FP32 inputs
    X, W = _data(N=1024, seed=5)
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=10, s_max=8, id_tol=1e-3, h=1.2))
    T.set_weights(W)
    U = T.evaluate()
    c = T.counts()
    perm = T.perm()
    X64 = X.astype(np.float64)
    for i in range(0, 1024, 53):
        nl, fl, _ = _lists(T, i)
        u = 0.0
        for a in nl:
            js = perm[c["start"][a]: c["start"][a] + c["size"][a]]
            u += np.exp(-0.5 * ((X64[js] - X64[i]) ** 2).sum(1) / H2) @ W[js, 0]
        for a in fl:
            nd = T.node(a)
            u += np.exp(-0.5 * ((X64[nd["skel"]] - X64[i]) ** 2).sum(1) / H2) @ nd["wsk"][:, 0]
        assert abs(u - U[i, 0]) <= 1e-12 * max(1.0, abs(u))


def _leaf_lists(T, a):
    """Near leaves and far nodes shared by the targets of leaf a in the
    leaf-grouped mode: U = ancestors of the leaves of every p in a and its
    neighbors."""
    ids, _ = T.knn()
    perm = T.perm()
    c = T.counts()
    L = T.L
    leafof = np.zeros(T.N, np.int64)
    for b in range(1 << L, 2 << L):
        leafof[perm[c["start"][b]: c["start"][b] + c["size"][b]]] = b
    members = perm[c["start"][a]: c["start"][a] + c["size"][a]]
    near = sorted({int(leafof[j]) for p in members for j in [p] + list(ids[p])})
    U = set()
    for lf in near:
        b = lf
        while b >= 1:
            U.add(b)
            b //= 2
    far = sorted({b ^ 1 for b in U if b > 1 and (b ^ 1) not in U})
    return near, far, leafof


def test_leaf_grouped_lists_list_form_and_counts():
    """Leaf-grouped lists (prune = 2): every target of a leaf is summed over
    the same Near leaves and Far skeletons, built here by set algebra from
    the union of the leaf's prune sets and summed with numpy."""
    H2 = float(np.float32(1.2)) ** 2
    X, W = _data(N=1024, seed=7)
    base = dict(leaf_size=32, kappa=6, s_max=8, id_tol=1e-3, h=1.2)
    T = oracle.Tree(X, oracle.Config(prune=2, **base))
    T.set_weights(W)
    U, near, far = T.evaluate(counts=True)
    T1 = oracle.Tree(X, oracle.Config(prune=1, **base))
    T1.set_weights(W)
    _, near1, far1 = T1.evaluate(counts=True)
    c = T.counts()
    perm = T.perm()
    X64 = X.astype(np.float64)
    for a in range(1 << T.L, 2 << T.L, 3):
        nl, fl, _ = _leaf_lists(T, a)
        members = perm[c["start"][a]: c["start"][a] + c["size"][a]]
        assert (near[members] == len(nl)).all() and (far[members] == len(fl)).all()
        assert (near[members] >= near1[members]).all()
        for i in members[::7]:
            u = 0.0
            for b in nl:
                js = perm[c["start"][b]: c["start"][b] + c["size"][b]]
                u += np.exp(-0.5 * ((X64[js] - X64[i]) ** 2).sum(1) / H2) @ W[js, 0]
            for b in fl:
                nd = T.node(b)
                u += np.exp(-0.5 * ((X64[nd["skel"]] - X64[i]) ** 2).sum(1) / H2) @ nd["wsk"][:, 0]
            assert abs(u - U[i, 0]) <= 1e-12 * max(1.0, abs(u))


def test_leaf_grouped_lists_are_at_least_as_accurate_here():
    """More of each target's sum is exact in the leaf-grouped mode: on this
    seeded mixture its error against the direct sum is below the per-target
    mode's (the same skeletons; only the lists differ)."""
    w = wl.SMALL_MIXTURE.scaled(2048)
    X, W = w.make_points(), w.make_weights().astype(np.float64)
    tg = np.arange(0, 2048, 4)
    ref = oracle.direct(X, W, 1.0, 0.5, targets=tg)
    errs = {}
    for pr in (1, 2):
        T = oracle.Tree(X, oracle.Config(leaf_size=64, kappa=4, s_max=8, id_tol=0.0, h=1.0, prune=pr))
        T.set_weights(W)
        errs[pr] = rel(T.evaluate(tg), ref)
    assert errs[2] < errs[1]


def test_linear_in_weights_and_multiple_rhs():
    X, W = _data(N=512, seed=6)
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=8, s_max=6, id_tol=1e-4, h=1.0))
    rng = np.random.default_rng(0)
    W2 = rng.standard_normal((512, 3))
    T.set_weights(W2)
    U = T.evaluate()
    for q in range(3):
        T.set_weights(W2[:, q:q + 1])
        assert np.allclose(T.evaluate()[:, 0], U[:, q], rtol=1e-12, atol=1e-12)


def test_error_falls_with_skeleton_size():
    w = wl.SMALL_MIXTURE.scaled(2048)
    X, W = w.make_points(), w.make_weights().astype(np.float64)
    tg = np.arange(0, 2048, 4)
    ref = oracle.direct(X, W, 1.0, 0.5, targets=tg)
    errs = []
    for s in (2, 8, 32):
        T = oracle.Tree(X, oracle.Config(leaf_size=64, kappa=8, s_max=s, id_tol=0.0, h=1.0))
        T.set_weights(W)
        errs.append(rel(T.evaluate(tg), ref))
    assert errs[0] > errs[1] > errs[2]


def test_out_of_sample_reductions():
    X, W = _data(N=512, seed=7)
    rng = np.random.default_rng(1)
    Y = (X[rng.integers(0, 512, 40)] + 0.1 * rng.standard_normal((40, 4))).astype(np.float32)
    ref = oracle.direct(X, W, 1.0, 0.5, Y=Y)
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=8, s_max=100000, id_tol=0.0, h=1.0))
    T.set_weights(W)
    U, knn, near, far = T.evaluate_oos(Y, counts=True)
    assert rel(U, ref) < 1e-13
    D = ((Y[:, None, :].astype(np.float64) - X[None].astype(np.float64)) ** 2).sum(-1)
    for q in range(40):
        assert np.array_equal(knn[q], np.lexsort((np.arange(512), D[q]))[:8])
    T0 = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=8, s_max=4, id_tol=0.0, h=1.0, prune=0))
    T0.set_weights(W)
    assert rel(T0.evaluate_oos(Y), ref) < 1e-13


def test_variable_bandwidth_kth_neighbor():
    X, W = _data(N=256, seed=8)
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=8, s_max=100000, id_tol=0.0, bw_mode=2, bw_k=4))
    ids, dd = oracle.knn_exact(X, 8)
    h = np.sqrt(dd[:, 3]).astype(np.float32)
    assert np.array_equal(T.hsrc(), h)
    T.set_weights(W)
    assert rel(T.evaluate(), oracle.direct(X, W, h, 0.5, targets=np.arange(256))) < 1e-13


def test_near_and_far_parts():
    """The near field alone (direct leaf sums, whose error is the paper's
    eps_kappa) and the far field alone (skeleton sums) add up to Evaluate;
    with pruning off the far field vanishes and the near field is the direct
    sum; the near field alone equals a brute-force sum over each target's
    near leaves (from the definition of U_i)."""
    X, W = _data(seed=4)
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=6, s_max=8, id_tol=0.0, h=1.0))
    T.set_weights(W)
    near, far, tot = T.evaluate_part("near"), T.evaluate_part("far"), T.evaluate()
    assert np.abs(near + far - tot).max() <= 1e-12 * np.abs(tot).max()
    assert np.abs(far).max() > 0 and np.abs(near).max() > 0
    perm = T.perm()
    c = T.counts()
    leaf_of = np.empty(len(X), np.int64)
    M = 1 << T.L
    for lf in range(M):
        a = M + lf
        leaf_of[perm[c["start"][a]: c["start"][a] + c["size"][a]]] = lf
    ids, _ = T.knn()
    for i in (0, 17, 300):
        leaves = {leaf_of[i]} | {leaf_of[j] for j in ids[i]}
        pts = np.concatenate([perm[c["start"][M + lf]: c["start"][M + lf] + c["size"][M + lf]] for lf in sorted(leaves)])
        D = ((X[i].astype(np.float64) - X[pts].astype(np.float64)) ** 2).sum(1)
        ref = (np.exp(-0.5 * D) * W[pts, 0]).sum()
        assert abs(near[i, 0] - ref) <= 1e-12 * (np.abs(W).sum())
    T0 = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=6, s_max=8, id_tol=0.0, h=1.0, prune=0))
    T0.set_weights(W)
    assert np.abs(T0.evaluate_part("far")).max() == 0.0
    assert rel(T0.evaluate_part("near"), oracle.direct(X, W, 1.0, 0.5, targets=np.arange(len(X)))) < 1e-13


def test_hit_rate():
    """hr (Section 4): the mean fraction of the exact neighbors found."""
    a = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    assert oracle.hit_rate(a, a) == 1.0
    assert oracle.hit_rate(a, a + 100) == 0.0
    b = np.array([[4, 3, 9, 1], [8, 0, 0, 0]])       # 3 of 4, then 1 of 4
    assert oracle.hit_rate(b, a) == (3 + 1) / 8
    X, _ = _data(N=400, seed=5)
    ex, _ = oracle.knn_exact(X, 8)
    rp, _ = oracle.knn_rp(X, 8, 1, 64, 3)
    rp_all, _ = oracle.knn_rp(X, 8, 1, 400, 3)        # one leaf holds every point: exact
    assert oracle.hit_rate(rp_all, ex) == 1.0
    assert 0.0 < oracle.hit_rate(rp, ex) < 1.0
