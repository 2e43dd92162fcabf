"""Autotuner: every candidate launch configuration is timed, exactly one is
kept, and the evaluation gives the same bits before and after tuning (the
configuration changes scheduling and staging, never the arithmetic)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,r,n_cand", [("fp16x3", 1, 8), ("fp16x3", 3, 8), ("bf16x3", 1, 2),
                                                ("simt_fp32", 1, 1)])
def test_autotune_keeps_results_and_picks_one(precision, r, n_cand):
    from paper_1410_0260_gb300 import askit, workloads
    w = workloads.MANIFOLD_1M_64.scaled(16384)
    X = torch.from_numpy(w.make_points()).cuda()
    t = askit.Tree(X, askit.Config(leaf_size=512, kappa=16, knn_mode=1, rp_iters=2, s_max=128, id_tol=1e-4,
                                   h=0.35, precision=precision))
    W = torch.from_numpy(np.random.default_rng(2).standard_normal((16384, r)).astype(np.float32)).cuda()
    t.set_weights(W)
    before = t.evaluate().clone()
    cands = t.autotune(reps=2)
    assert len(cands) == n_cand
    assert sum(c["chosen"] for c in cands) == 1
    assert all(c["ms"] > 0 for c in cands)
    best = min(cands, key=lambda c: c["ms"])
    assert best["chosen"]
    after = t.evaluate()
    torch.cuda.synchronize()
    assert torch.equal(before, after)
    t.close()


def test_autotune_needs_weights():
    from paper_1410_0260_gb300 import askit
    t = askit.Tree(torch.randn((2048, 8), device="cuda"), askit.Config(leaf_size=128, kappa=8, s_max=16))
    with pytest.raises(askit.AskitError):
        t.autotune()
    t.close()
