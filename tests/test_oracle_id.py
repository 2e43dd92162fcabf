"""Pins for the interpolative decomposition by pivoted QR (Section 2.1,
eq. (2.1)): pivots against scipy's pivoted QR, the paper's error bound
against numpy's SVD, exact low-rank recovery, and the skeleton-weight
identity K(T, C) v - K(T, S) w~ = (K_R - K_S P) v_R."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle


def test_pivots_match_scipy_on_separated_norms():
    rng = np.random.default_rng(0)
    rows, cols = 60, 30
    scales = 1.7 ** -rng.permutation(cols)
    A = rng.standard_normal((rows, cols)) * scales
    piv, P, s, rd = oracle.cpqr_id(A, 0.0, cols, cols)
    _, R, p_ref = sla.qr(A, pivoting=True, mode="economic")
    assert s == cols
    assert list(piv) == list(p_ref)
    assert np.allclose(np.abs(rd), np.abs(np.diag(R)), rtol=1e-10)


def test_rdiag_nonincreasing_and_r00_is_max_column_norm():
    rng = np.random.default_rng(1)
    A = rng.standard_normal((40, 25))
    piv, P, s, rd = oracle.cpqr_id(A, 0.0, 25, 25)
    assert (np.diff(np.abs(rd)) <= 1e-12).all()
    assert abs(abs(rd[0]) - np.linalg.norm(A, axis=0).max()) < 1e-12


@pytest.mark.parametrize("s", [3, 8, 15])
def test_paper_error_bound(s):
    rng = np.random.default_rng(2 + s)
    rows, cols = 70, 40
    U, _ = np.linalg.qr(rng.standard_normal((rows, cols)))
    V, _ = np.linalg.qr(rng.standard_normal((cols, cols)))
    sig = 0.6 ** np.arange(cols)
    A = (U * sig) @ V.T
    piv, P, got, _ = oracle.cpqr_id(A, 0.0, s, s)
    assert got == s
    AS, AR = A[:, piv[:s]], A[:, piv[s:]]
    err = np.linalg.norm(AR - AS @ P, 2)
    sv = np.linalg.svd(A, compute_uv=False)
    assert err <= np.sqrt(1 + cols * (cols - s)) * sv[s]


def test_exact_low_rank_is_recovered():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((50, 5)) @ rng.standard_normal((5, 30))
    piv, P, s, _ = oracle.cpqr_id(A, 1e-10, 1, 30)
    assert s == 5
    err = np.linalg.norm(A[:, piv[5:]] - A[:, piv[:5]] @ P)
    assert err <= 1e-12 * np.linalg.norm(A)


def test_rank_clamps():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((20, 12))
    assert oracle.cpqr_id(A, 0.9, 4, 10)[2] >= 4          # s_min wins over the tolerance
    assert oracle.cpqr_id(A, 0.0, 1, 6)[2] == 6           # s_max caps
    assert oracle.cpqr_id(A[:5], 0.0, 1, 12)[2] == 5      # never more than the rows
    assert oracle.cpqr_id(np.zeros((6, 4)), 0.5, 2, 4)[2] == 0   # an all-zero block has no skeleton


def test_skeleton_weight_identity_on_tree_nodes():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((256, 3)).astype(np.float32)
    cfg = oracle.Config(leaf_size=32, kappa=6, s_max=8, id_tol=0.0, h=0.9)
    T = oracle.Tree(X, cfg)
    W = rng.standard_normal((256, 2))
    T.set_weights(W)
    X64 = X.astype(np.float64)
    for a in range(1 << T.L, 2 << T.L):          # leaves: v = w(X_a)
        nd = T.node(a)
        Tr, Cc, S, s = nd["trows"], nd["cols"], nd["skel"], len(nd["skel"])
        K = np.exp(-0.5 * ((X64[Tr][:, None] - X64[Cc][None]) ** 2).sum(-1) / float(np.float32(0.9)) ** 2)
        KS = K[:, nd["piv"][:s]]
        KR = K[:, nd["piv"][s:]]
        v = W[Cc]
        lhs = K @ v - KS @ nd["wsk"]
        rhs = (KR - KS @ nd["P"]) @ v[nd["piv"][s:]]
        assert np.allclose(lhs, rhs, atol=1e-12)
        assert list(S) == list(Cc[nd["piv"][:s]])


def test_householder_sign_convention():
    # beta = -sign(alpha) ||x||: R_kk carries the sign opposite to the pivot's leading entry
    rng = np.random.default_rng(6)
    for _ in range(20):
        A = rng.standard_normal((12, 7))
        piv, P, s, rd = oracle.cpqr_id(A, 0.0, 1, 1)
        assert np.sign(rd[0]) == -np.sign(A[0, piv[0]])


def test_pivot_ties_take_the_smallest_position():
    rng = np.random.default_rng(7)
    a = rng.standard_normal(10) * 5
    A = np.stack([rng.standard_normal(10), a, rng.standard_normal(10), a.copy(), a[::-1].copy()], 1)
    piv, P, s, rd = oracle.cpqr_id(A, 0.0, 1, 1)
    assert piv[0] == 1          # columns 1, 3 and 4 tie on the largest norm


def test_node_ids_approximate_the_true_kernel_block():
    """The ID of every node is an ID of K(T_a, C_a) built with the paper's
    Gaussian exp(-c r^2 / h^2) (Section 4): its error obeys eq. (2.1)."""
    rng = np.random.default_rng(8)
    X = rng.standard_normal((512, 3)).astype(np.float32)
    h = 0.7
    cfg = oracle.Config(leaf_size=32, kappa=6, s_max=6, id_tol=0.0, h=h)
    T = oracle.Tree(X, cfg)
    X64 = X.astype(np.float64)
    h2 = float(np.float32(h)) ** 2
    checked = 0
    for a in range(2, 2 << T.L):
        nd = T.node(a)
        s, c = len(nd["skel"]), len(nd["cols"])
        if s == c or s == 0:
            continue
        K = np.exp(-0.5 * ((X64[nd["trows"]][:, None] - X64[nd["cols"]][None]) ** 2).sum(-1) / h2)
        err = np.linalg.norm(K[:, nd["piv"][s:]] - K[:, nd["piv"][:s]] @ nd["P"], 2)
        sv = np.linalg.svd(K, compute_uv=False)
        assert err <= np.sqrt(1 + c * (c - s)) * sv[s] + 1e-13, a
        checked += 1
    assert checked > 10


def test_node_pivots_match_scipy_on_true_kernel_block():
    """Leading pivots of each node's ID equal scipy's pivoted QR of the block
    K(T_a, C_a) formed with exp(-c r^2 / h^2) (checked where the pivot norms
    are well separated, so the rounding of norm downdating cannot decide)."""
    rng = np.random.default_rng(10)
    X = rng.standard_normal((512, 3)).astype(np.float32)
    h = 0.6
    T = oracle.Tree(X, oracle.Config(leaf_size=32, kappa=6, s_max=8, id_tol=0.0, h=h))
    X64 = X.astype(np.float64)
    h2 = float(np.float32(h)) ** 2
    compared = 0
    for a in range(2, 2 << T.L):
        nd = T.node(a)
        s = len(nd["skel"])
        K = np.exp(-0.5 * ((X64[nd["trows"]][:, None] - X64[nd["cols"]][None]) ** 2).sum(-1) / h2)
        _, R, p_ref = sla.qr(K, pivoting=True, mode="economic")
        rd = np.abs(np.diag(R))
        for q in range(min(s, 4)):
            if q + 1 < len(rd) and rd[q + 1] > rd[q] * (1 - 1e-6):
                break
            assert nd["piv"][q] == p_ref[q], (a, q)
            compared += 1
    assert compared > 40
