"""Exact kNN of new points against a tree's points (the tensor-core shortlist
with the FP64 re-rank, and its exhaustive fallback) against the FP64 oracle's
exact kNN: identical ids and bitwise identical FP64 distances."""
import numpy as np
import pytest

import oracle
from paper_1410_0260_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tree(X, **kw):
    from paper_1410_0260_gb300 import askit
    return askit.Tree(torch.from_numpy(X).cuda(), askit.Config(**kw))


def _check(tree, X, Y, kappa):
    ids, dist = tree.knn_targets(torch.from_numpy(Y).cuda())
    oid, odd = oracle.knn_exact(X, kappa, Y=Y)
    assert np.array_equal(ids.cpu().numpy(), oid)
    assert np.array_equal(dist.cpu().numpy(), odd)


def test_manifold_queries_match_the_oracle():
    w = wl.SERVING_2M_64.scaled(32768)
    X = w.make_points()
    t = _tree(X, leaf_size=512, kappa=32, knn_mode=1, rp_iters=2, s_max=64, id_tol=1e-3, h=0.4, seed=5)
    Y = wl.manifold_queries(3000, w.d, w.k_intr, w.noise, w.seed, 123)
    _check(t, X, Y, 32)
    t.close()


def test_ragged_tree_far_queries_and_small_d():
    X = wl.mixture(5000, 12, 4, 3.0, seed=41)
    t = _tree(X, leaf_size=100, kappa=10, knn_mode=0, s_max=16, h=2.0, seed=2)
    rng = np.random.default_rng(3)
    Y = np.concatenate([X[rng.integers(0, 5000, 300)] + 0.1 * rng.standard_normal((300, 12)),
                        rng.uniform(-20, 20, (77, 12))]).astype(np.float32)    # some far from the data
    _check(t, X, Y, 10)
    t.close()


def test_duplicates_overflow_the_shortlist_and_fall_back():
    """2000 copies of one point: a query next to it has more than 1024 sources
    within its bound, so it takes the exhaustive search; ties break by id."""
    rng = np.random.default_rng(8)
    X = np.concatenate([rng.standard_normal((6000, 16)),
                        np.repeat(rng.standard_normal((1, 16)), 2000, axis=0)]).astype(np.float32)
    t = _tree(X, leaf_size=256, kappa=16, knn_mode=0, s_max=16, h=1.0, seed=4)
    Y = np.concatenate([X[-1:] + 1e-3, X[:50] + 0.05]).astype(np.float32)
    _check(t, X, Y, 16)
    t.close()
