"""Serving loop: each request's result is the same alone and in a mixed,
continuously batched stream (weight requests merged column-wise, target
batches concatenated, two slots overlapping on the device), and admission by
memory footprint rejects what can never fit.

The plain FP32 path computes every target's sum independently of the other
targets, so its results are bit-identical alone and in the mix.  So is FP16x3
for target batches: every row's terms are formed the same way at any
position of its item.  A weight request takes the form its batch's number of
vectors selects (one vector, up to four summed on the FP32 pipe, more on the
tensor cores), and alone it may take another form than merged, so weight
requests are held to the split-path tolerance (relative L2 1e-4): a result
routed to the wrong request would be off by order one."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _tree(precision="fp16x3"):
    from paper_1410_0260_gb300 import askit, workloads
    w = workloads.SERVING_2M_64.scaled(8192)
    X = w.make_points()
    cfg = askit.Config(leaf_size=256, kappa=16, knn_mode=0, s_max=64, id_tol=1e-4, h=0.4, precision=precision)
    return askit.Tree(torch.from_numpy(X).cuda(), cfg), X


def _requests(X, rng):
    from paper_1410_0260_gb300.serve import Request
    N, d = X.shape
    reqs = []
    for k in range(12):
        if k % 2 == 0:
            r = int(rng.integers(1, 7))
            reqs.append(Request("weights", torch.from_numpy(rng.standard_normal((N, r)).astype(np.float32))))
        else:
            T = int(rng.integers(20, 300))
            Y = X[rng.integers(0, N, T)] + 0.05 * rng.standard_normal((T, d)).astype(np.float32)
            reqs.append(Request("targets", torch.from_numpy(Y.astype(np.float32))))
    return reqs


@pytest.mark.parametrize("precision", ["simt_fp32", "fp16x3"])
def test_results_alone_equal_results_in_the_mix(precision):
    from paper_1410_0260_gb300.serve import Request, Server
    tree, X = _tree(precision)
    rng = np.random.default_rng(0)
    Wres = torch.from_numpy(rng.standard_normal((X.shape[0], 2)).astype(np.float32))
    reqs = _requests(X, rng)
    # alone: one request at a time
    srv = Server(tree, Wres, n_slots=1)
    alone = []
    for r in reqs:
        q = srv.submit(Request(r.kind, r.data))
        assert q.done.wait(60), "request not answered"
        assert q.error is None, q.error
        alone.append(q.result.clone())
    srv.close()
    # mixed: everything at once, two slots, continuous batching
    srv = Server(tree, Wres, n_slots=2)
    mixed = [srv.submit(Request(r.kind, r.data)) for r in reqs]
    for q in mixed:
        assert q.done.wait(120), "request not answered"
        assert q.error is None, q.error
    completed = len(srv.completed)
    n_batches, peak = srv.n_batches, srv.peak_concurrency
    srv.close()
    assert completed == len(mixed)
    # continuous batching, not a queue: requests were merged into fewer
    # batches than requests, and two batches were on the device at once
    assert n_batches < len(mixed), n_batches
    assert peak == 2, peak
    for a, q in zip(alone, mixed):
        b = q.result
        assert a.shape == b.shape
        if precision == "simt_fp32" or q.kind == "targets":
            assert torch.equal(a, b), (q.kind, a.shape)
        else:
            rel = float(torch.linalg.vector_norm(a.double() - b.double()) / torch.linalg.vector_norm(a.double()))
            assert rel <= 1e-4, (q.kind, rel)
    tree.close()


def test_admission_by_footprint():
    from paper_1410_0260_gb300.serve import Request, Server, batch_bytes
    tree, X = _tree()
    Wres = torch.ones((X.shape[0], 1))
    small = batch_bytes(tree, "weights", 1)
    assert batch_bytes(tree, "weights", 16) > 1.5 * small
    # a budget that holds one single-vector weight batch but not a 16-vector one
    srv = Server(tree, Wres, n_slots=2, budget_bytes=int(small * 1.5))
    ok = srv.submit(Request("weights", torch.ones((X.shape[0], 1))))
    big = srv.submit(Request("weights", torch.ones((X.shape[0], 16))))
    ok.done.wait(60)
    big.done.wait(60)
    srv.close()
    assert ok.error is None
    assert big.error is not None and "budget" in big.error
    tree.close()
