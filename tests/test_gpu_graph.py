"""A captured set_weights + Evaluate step replays to the same bits as the
eager calls, and every replay reads the current contents of the bound W."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,r", [("fp16x3", 1), ("tf32x3", 3), ("simt_fp32", 2)])
def test_graph_replay_matches_eager_calls(precision, r):
    from paper_1410_0260_gb300 import askit, workloads
    w = workloads.MANIFOLD_1M_64.scaled(8192)
    X = torch.from_numpy(w.make_points()).cuda()
    t = askit.Tree(X, askit.Config(leaf_size=256, kappa=16, knn_mode=1, rp_iters=2, s_max=64, id_tol=1e-4,
                                   h=0.35, precision=precision))
    rng = np.random.default_rng(5)
    W = torch.from_numpy(rng.standard_normal((8192, r)).astype(np.float32)).cuda()
    U = torch.empty((8192, r), device="cuda")
    g = t.capture(W, U)
    for k in range(3):
        W.copy_(torch.from_numpy(rng.standard_normal((8192, r)).astype(np.float32)))
        g.launch()
        t.set_weights(W)
        ref = t.evaluate()
        torch.cuda.synchronize()
        assert torch.equal(U, ref), k
    g.close()
    t.close()


def test_graph_rejects_copied_buffers():
    from paper_1410_0260_gb300 import askit
    t = askit.Tree(torch.randn((512, 4), device="cuda"), askit.Config(leaf_size=64, kappa=8, s_max=8))
    W = torch.randn((2, 512), device="cuda").t()          # column-major view: would need a copy
    with pytest.raises(askit.AskitError):
        t.capture(W, torch.empty((512, 2), device="cuda"))
    t.close()
