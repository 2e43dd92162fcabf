"""Pins for the oracle's counter RNG (Philox4x64-10) and canonical exp.

The sampling rule of eq. (2.4) and the random-projection directions draw from
Philox; the ID's kernel matrices use the canonical exp.  Both are pinned to
outside definitions: the published Philox known-answer vectors, numpy's
Philox bit generator, and mpmath's exp.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden", "philox4x64_10_kat.txt")


def _kat():
    rows = []
    for line in open(GOLD):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,out", _kat())
def test_philox_known_answers(ctr, key, out):
    got = oracle.philox4x64_10(ctr, key)
    assert [int(x) for x in got] == out


def test_philox_matches_numpy_stream():
    rng = np.random.default_rng(7)
    for _ in range(50):
        ctr = [int(x) for x in rng.integers(0, 2**63, size=4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.uint64)]
        c = sum(v << (64 * i) for i, v in enumerate(ctr))
        k = sum(v << (64 * i) for i, v in enumerate(key))
        # numpy's Philox advances its counter before producing a block
        bg = np.random.Philox(key=k, counter=(c - 1) % (1 << 256))
        assert (oracle.philox4x64_10(ctr, key) == bg.random_raw(4)).all()


def _ulps(a, b):
    return abs(a - b) / math.ulp(b) if b != 0 else abs(a) / 5e-324


def test_cexp_within_two_ulp_of_mpmath():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.prec = 120
    rng = np.random.default_rng(3)
    args = np.concatenate([-rng.uniform(0, 1, 400), -rng.uniform(0, 50, 400),
                           -rng.uniform(0, 699, 400), [0.0, -1e-300, -0.5, -math.log(2), -700.0]])
    worst = 0.0
    for a in args:
        exact = float(mpmath.exp(mpmath.mpf(float(a))))
        worst = max(worst, _ulps(oracle.cexp(a), exact))
    assert worst <= 2.0, worst


def test_cexp_special_values():
    assert oracle.cexp(0.0) == 1.0
    assert oracle.cexp(-701.0) == 0.0
    # monotone on a fine grid crossing many reduction intervals
    grid = np.linspace(-60.0, 0.0, 20001)
    vals = np.array([oracle.cexp(a) for a in grid])
    assert (np.diff(vals) >= 0).all()
    # exp(a) exp(b) = exp(a + b) with a + b exact (integers)
    for a, b in [(-3.0, -4.0), (-100.0, -200.0), (-0.0, -17.0)]:
        assert abs(oracle.cexp(a) * oracle.cexp(b) / oracle.cexp(a + b) - 1.0) < 1e-15
