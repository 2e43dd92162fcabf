"""Pins for node neighbor lists (Algorithm 2 with the truncation of Section
2.2) and the sampled skeletonization targets (eq. (2.4)), by brute-force set
algebra and an independent replay of the sampling rule on numpy's Philox."""
import numpy as np
import pytest

import oracle


@pytest.fixture(scope="module")
def small_tree():
    rng = np.random.default_rng(11)
    X = (rng.standard_normal((512, 4)) + rng.integers(0, 3, (512, 1)) * 4).astype(np.float32)
    cfg = oracle.Config(leaf_size=32, kappa=8, s_max=10, ell_extra=6, id_tol=1e-8, h=1.0, seed=77)
    return X, cfg, oracle.Tree(X, cfg)


def leaf_ranges(T):
    c = T.counts()
    L = T.L
    return c, {a: set(T.perm()[c["start"][a]: c["start"][a] + c["size"][a]])
               for a in range(1, 2 << L)}


def test_node_lists_brute_force(small_tree):
    X, cfg, T = small_tree
    ids, dd = T.knn()
    c, members = leaf_ranges(T)
    ell = cfg.s_max + cfg.ell_extra
    L = T.L
    lists = {}
    for depth in range(L, 0, -1):
        for a in range(1 << depth, 2 << depth):
            key = {}
            if depth == L:
                for i in members[a]:
                    for j, D in zip(ids[i], dd[i]):
                        if j in members[a]:
                            continue
                        key[j] = min(key.get(j, np.inf), D)
            else:
                for ch in (2 * a, 2 * a + 1):
                    for j, D in lists[ch]:
                        if j in members[a]:
                            continue
                        key[j] = min(key.get(j, np.inf), D)
            lst = sorted(key.items(), key=lambda kv: (kv[1], kv[0]))[:ell]
            lists[a] = lst
            node = T.node(a)
            assert [j for j, _ in lst] == list(node["nl_ids"]), a
            assert np.array_equal([k for _, k in lst], node["nl_key"]), a


def test_sampled_targets_replayed_on_numpy_philox(small_tree):
    X, cfg, T = small_tree
    c, members = leaf_ranges(T)
    N = X.shape[0]
    ellmax = cfg.s_max + cfg.ell_extra
    for a in range(2, 2 << T.L):
        node = T.node(a)
        ell = min(ellmax, N - len(members[a]))
        rows = list(node["nl_ids"][:ell])
        bg = None
        n = 0
        buf = []
        while len(rows) < ell:
            if n % 4 == 0:
                # stream keyed (seed, 0), block (a, n/4, 0, 0); numpy advances before drawing
                ctr = a + ((n // 4) << 64)
                bg = np.random.Philox(key=cfg.seed, counter=ctr - 1)
                buf = list(bg.random_raw(4))
            w = int(buf[n % 4])
            n += 1
            j = ((w >> 32) * N) >> 32
            if j in members[a] or j in rows:
                continue
            rows.append(j)
        assert rows == list(node["trows"]), a
        assert len(set(rows)) == ell and not (set(rows) & members[a])
