"""Host logic of the serving loop, on the CPU with a stand-in tree: batching
(weight requests merged column-wise and evaluated in chunks, target batches
concatenated), routing of each request's slice of the batch result,
admission by footprint, rejection of what can never fit, and identity of
requests (two equal-looking requests stay distinct).  The stand-in computes a
simple function of its inputs so that every routed slice can be checked."""
import threading
import time

import numpy as np
import pytest
import torch

from paper_1410_0260_gb300.serve import Request, Server, batch_bytes, latency_stats, replay


class _Ctx:
    def __init__(self, tree):
        self.tree, self.r, self.W = tree, 0, None

    def set(self, W, stream=None):
        assert W.shape[1] <= 16          # evaluations stay within the chunk width
        self.W, self.r = W.clone(), W.shape[1]
        self.tree.calls.append(("set", W.shape[1]))

    def evaluate(self, stream=None):
        time.sleep(0.002)
        return 2.0 * self.W + torch.arange(self.tree.N, dtype=torch.float32)[:, None]

    def evaluate_targets(self, Y, stream=None):
        time.sleep(0.002)
        self.tree.calls.append(("targets", Y.shape[0]))
        return Y.sum(1, keepdim=True) * self.W.sum()

    def close(self):
        pass


class _Tree:
    def __init__(self, N=64, d=3):
        self.N, self.d, self.device, self.calls = N, d, torch.device("cpu"), []

    def weights_context(self):
        return _Ctx(self)

    def footprint(self, kind, n, r):
        return 1000 * r if kind == 0 else 10 * n + 100


def _expect_weights(tree, W):
    return 2.0 * W + torch.arange(tree.N, dtype=torch.float32)[:, None]


def test_batching_and_routing():
    tree = _Tree()
    Wres = torch.ones((tree.N, 1))
    srv = Server(tree, Wres, n_slots=2, budget_bytes=10 ** 9)
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(30):
        if k % 3:
            W = torch.from_numpy(rng.standard_normal((tree.N, int(rng.integers(1, 40)))).astype(np.float32))
            reqs.append(srv.submit(Request("weights", W)))
        else:
            Y = torch.from_numpy(rng.standard_normal((int(rng.integers(1, 50)), tree.d)).astype(np.float32))
            reqs.append(srv.submit(Request("targets", Y)))
    for r in reqs:
        assert r.done.wait(30)
        assert r.error is None, r.error
        if r.kind == "weights":
            assert torch.equal(r.result, _expect_weights(tree, r.data))
        else:
            assert torch.allclose(r.result, r.data.sum(1, keepdim=True) * tree.N)
    srv.close()
    assert srv.n_batches < len(reqs)                   # something was merged
    assert max(n for c, n in tree.calls if c == "set") <= 16


def test_identical_requests_stay_distinct():
    tree = _Tree()
    srv = Server(tree, torch.ones((tree.N, 1)), n_slots=1, budget_bytes=10 ** 9)
    W = torch.ones((tree.N, 2))
    reqs = [srv.submit(Request("weights", W)) for _ in range(5)]
    for r in reqs:
        assert r.done.wait(30) and r.error is None
        assert torch.equal(r.result, _expect_weights(tree, W))
    srv.close()
    assert len({id(r) for r in srv.completed}) == 5


def test_admission_waits_and_rejects():
    tree = _Tree()
    srv = Server(tree, torch.ones((tree.N, 1)), n_slots=2,
                 budget_bytes=batch_bytes(tree, "weights", 16) + 10)
    ok = [srv.submit(Request("weights", torch.ones((tree.N, 16)))) for _ in range(3)]
    big = srv.submit(Request("targets", torch.ones((10 ** 6, tree.d))))
    for r in ok:
        assert r.done.wait(30) and r.error is None
    assert big.done.wait(30) and "budget" in big.error
    srv.close()
    assert srv.peak_concurrency == 1      # the budget holds one 16-column batch at a time


def test_replay_and_stats():
    tree = _Tree()
    srv = Server(tree, torch.ones((tree.N, 1)), n_slots=2, budget_bytes=10 ** 9)
    stream = [(0.001 * i, "weights" if i % 2 else "targets",
               torch.ones((tree.N, 3)) if i % 2 else torch.ones((7, tree.d))) for i in range(12)]
    reqs = replay(srv, stream, timeout=30)
    st = latency_stats(reqs, tree.N)
    srv.close()
    assert st["completed"] == 12 and st["p99_ms"] >= st["p50_ms"] > 0
    assert st["targets_per_s"] > 0


def test_scheduler_failure_fails_waiting_requests(monkeypatch):
    tree = _Tree()
    srv = Server(tree, torch.ones((tree.N, 1)), n_slots=1, budget_bytes=10 ** 9)
    def boom(*a, **k):
        raise RuntimeError("planted")
    monkeypatch.setattr(srv, "_take_batch", boom)
    r = srv.submit(Request("weights", torch.ones((tree.N, 1))))
    assert r.done.wait(30)
    assert "scheduler failed" in r.error
    srv.close()
