"""Pins for the oracle's direct sum, eq. (1.1), with the Gaussian of Section 4.

Closed forms: K(x, x) = 1, two-point sums written out by hand, linearity in
w, the source point's bandwidth (not the target's) in the variable-h kernel,
and the small-bandwidth limit u -> w.
"""
import math

import numpy as np

import oracle


def test_single_point_returns_weight():
    X = np.array([[0.3, -1.2, 4.0]], np.float32)
    W = np.array([[2.5, -1.0]])
    U = oracle.direct(X, W, 0.7, 0.5, targets=[0])
    assert np.array_equal(U, W)


def test_two_points_closed_form():
    X = np.array([[0.0, 0.0], [3.0, 4.0]], np.float32)     # distance^2 = 25
    W = np.array([[1.5], [-2.0]])
    h, c = 2.0, 0.5
    U = oracle.direct(X, W, h, c, targets=[0, 1])
    k = math.exp(-c * 25.0 / (h * h))
    assert abs(U[0, 0] - (1.5 + k * -2.0)) < 1e-15
    assert abs(U[1, 0] - (-2.0 + k * 1.5)) < 1e-15


def test_variable_bandwidth_uses_source_point():
    X = np.array([[0.0], [1.0]], np.float32)
    W = np.array([[1.0], [1.0]])
    h = np.array([1.0, 2.0], np.float32)
    U = oracle.direct(X, W, h, 1.0, targets=[0, 1])
    assert abs(U[0, 0] - (1.0 + math.exp(-1.0 / 4.0))) < 1e-15   # source 1 has h = 2
    assert abs(U[1, 0] - (1.0 + math.exp(-1.0 / 1.0))) < 1e-15   # source 0 has h = 1


def test_linear_in_weights():
    rng = np.random.default_rng(0)
    X = rng.standard_normal((200, 5)).astype(np.float32)
    W1, W2 = rng.standard_normal((200, 1)), rng.standard_normal((200, 1))
    t = np.arange(0, 200, 7)
    U1 = oracle.direct(X, W1, 0.8, 0.5, targets=t)
    U2 = oracle.direct(X, W2, 0.8, 0.5, targets=t)
    U12 = oracle.direct(X, 2.0 * W1 - 3.0 * W2, 0.8, 0.5, targets=t)
    assert np.allclose(U12, 2.0 * U1 - 3.0 * U2, rtol=1e-12, atol=1e-12)


def test_small_bandwidth_limit():
    X = (np.arange(20, dtype=np.float32) * 10.0).reshape(-1, 1)
    W = np.linspace(-1, 1, 20).reshape(-1, 1)
    U = oracle.direct(X, W, 0.1, 0.5, targets=np.arange(20))
    assert np.array_equal(U, W)


def test_out_of_sample_targets():
    X = np.array([[0.0, 0.0], [0.0, 2.0]], np.float32)
    W = np.array([[1.0], [3.0]])
    Y = np.array([[0.0, 1.0]], np.float32)
    U = oracle.direct(X, W, 1.0, 0.5, Y=Y)
    assert abs(U[0, 0] - 4.0 * math.exp(-0.5)) < 1e-15
