"""Pins for the oracle's refinements of the pruning that Section 3 proposes
(level-restricted far field, adaptive per-point kappa_i), checked against
what the definitions fix: the unrestricted cases reproduce Algorithm 4 bit
for bit, the Near/Far counts follow from brute-force set algebra on U_i, a
height limit of zero covers every leaf exactly once, a zero kappa_i leaves
only the target's own leaf, and kappa_i itself follows from the kernel
values at the neighbor distances."""
import numpy as np

import oracle


def _tree(N=1024, d=4, seed=0, **kw):
    rng = np.random.default_rng(seed)
    X = (rng.standard_normal((N, d)) + rng.integers(0, 4, (N, 1)) * 3.0).astype(np.float32)
    W = rng.standard_normal((N, 1))
    cfg = dict(leaf_size=32, kappa=8, s_max=6, id_tol=0.0, h=0.8)
    cfg.update(kw)
    T = oracle.Tree(X, oracle.Config(**cfg))
    T.set_weights(W)
    return X, W, T


def _leaf_of(T):
    perm, c = T.perm(), T.counts()
    M = 1 << T.L
    leaf = np.empty(T.N, np.int64)
    for lf in range(M):
        leaf[perm[c["start"][M + lf]: c["start"][M + lf] + c["size"][M + lf]]] = lf
    return leaf


def _brute_counts(T, i, far_height, kappa_i=None):
    """Near/Far of target i from the definition: U_i = ancestors of the
    leaves of {i} U N_i[:kappa_i]; Near = leaves in U_i; a node beta is far
    when it is not in U_i and either its parent is in U_i and beta is at most
    far_height above the leaves, or beta sits exactly far_height above the
    leaves and its parent (higher) is not used for a skeleton."""
    L = T.L
    ids, _ = T.knn()
    leaf = _leaf_of(T)
    k = ids.shape[1] if kappa_i is None else kappa_i
    leaves = {leaf[i]} | {leaf[j] for j in ids[i, :k]}
    U = set()
    for lf in leaves:
        a = (1 << L) + lf
        while a >= 1:
            U.add(a)
            a >>= 1
    near = len(leaves)
    far = 0
    fh = L if far_height < 0 else far_height
    for depth in range(1, L + 1):
        for b in range(1 << depth, 2 << depth):
            if b in U or L - depth > fh:
                continue
            # the normal rule (parent in U_i), or at the limit height a node
            # whose higher ancestor would have been pruned
            if (b >> 1) in U or L - depth == fh:
                far += 1
    return near, far


def test_unrestricted_cases_are_algorithm_4():
    X, W, T = _tree()
    U = T.evaluate()
    assert np.array_equal(T.evaluate_ext(-1, 0.0), U)
    assert np.array_equal(T.evaluate_ext(T.L - 1, 0.0), U)        # every non-root node is allowed
    assert np.array_equal(T.evaluate_ext(-1, 1e300), U)           # every neighbor kept


def test_level_restricted_counts_follow_the_definition():
    X, W, T = _tree(seed=1)
    for fh in (0, 1, 2, T.L - 2):
        _, near, far = T.evaluate_ext(fh, 0.0, counts=True)
        for i in (0, 5, 777, T.N - 1):
            assert (near[i], far[i]) == _brute_counts(T, i, fh), (fh, i)
    _, near, far = T.evaluate_ext(0, 0.0, counts=True)
    assert (near + far == (1 << T.L)).all()                        # height 0: every leaf, once


def test_height_zero_with_full_skeletons_is_the_direct_sum():
    X, W, T = _tree(seed=2, s_max=100000)
    U = T.evaluate_ext(0, 0.0)
    ref = oracle.direct(X, W, 0.8, 0.5, targets=np.arange(len(X)))
    assert np.linalg.norm(U - ref) / np.linalg.norm(ref) < 1e-12


def test_adaptive_kappa():
    X, W, T = _tree(seed=3)
    ids, dd = T.knn()
    # kappa_i = 0 everywhere: only the own leaf is near, one far node per level
    _, near, far = T.evaluate_ext(-1, 1e-300, counts=True)
    assert (near == 1).all() and (far == T.L).all()
    # kappa_i from the kernel values at the neighbor distances (constant h)
    cut = 3.0
    arg = 0.5 * dd / (np.float32(0.8).astype(np.float64) ** 2)
    kap = np.array([1 + max([z for z in range(ids.shape[1]) if arg[i, z] < cut], default=-1) for i in range(T.N)])
    assert kap.min() < ids.shape[1] and kap.max() > 0              # the cut bites on this data
    _, near, far = T.evaluate_ext(-1, cut, counts=True)
    for i in (0, 11, 400, T.N - 1):
        assert (near[i], far[i]) == _brute_counts(T, i, -1, kappa_i=int(kap[i])), i
    # a looser cut keeps at least as many neighbors, so it prunes no more
    _, near2, _ = T.evaluate_ext(-1, 2 * cut, counts=True)
    assert (near2 >= near).all()
