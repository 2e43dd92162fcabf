"""Autotuner and launch configurations: every candidate is timed and exactly
one kept; schedules, stages and tiled runs change no result bit; paired
256-column items (which sum both sub-blocks' columns in one accumulator)
agree to FP32 rounding; every configuration matches the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


# candidates: FP16x3 with global centering (the automatic choice here) has
# two schedules x stages 3, 4 + paired items at stages 3, 4 (none past
# r = 4); per sub-block centering two schedules x stages 2, 3 x tiled runs
# on/off + paired items with tiled runs on/off
@pytest.mark.parametrize("precision,centering,r,n_cand",
                         [("fp16x3", "auto", 1, 6), ("fp16x3", "auto", 3, 6), ("fp16x3", "auto", 6, 4),
                          ("fp16x3", "block", 1, 10), ("fp16x3", "block", 3, 10), ("fp16x3", "block", 6, 8),
                          ("bf16x3", "auto", 1, 2), ("simt_fp32", "auto", 1, 1)])
def test_autotune_keeps_results_and_picks_one(precision, centering, r, n_cand):
    from paper_1410_0260_gb300 import askit, workloads
    w = workloads.MANIFOLD_1M_64.scaled(16384)
    X = torch.from_numpy(w.make_points()).cuda()
    t = askit.Tree(X, askit.Config(leaf_size=512, kappa=16, knn_mode=1, rp_iters=2, s_max=128, id_tol=1e-4,
                                   h=0.35, precision=precision))
    t.set_fp16_centering(centering)
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
    if best.get("pairs"):
        rel = float(torch.linalg.vector_norm((before - after).double()) / torch.linalg.vector_norm(before.double()))
        assert rel <= 1e-6
    else:
        assert torch.equal(before, after)
    t.close()


def test_every_launch_configuration_matches_the_oracle():
    import oracle
    from paper_1410_0260_gb300 import askit, workloads
    w = workloads.MANIFOLD_1M_64.scaled(8192)
    X = w.make_points()
    kw = dict(leaf_size=512, kappa=16, knn_mode=1, rp_iters=2, s_max=200, id_tol=1e-4, h=0.35, seed=3)
    ot = oracle.Tree(X, oracle.Config(**kw))
    gt = askit.Tree(torch.from_numpy(X).cuda(), askit.Config(precision="fp16x3", **kw))
    for r, centering in ((1, "auto"), (3, "auto"), (1, "block"), (3, "block")):
        gt.set_fp16_centering(centering)
        # the split-path tolerance for the global centering, FP32 grade per block
        tol = 1e-4 if centering == "auto" else 1e-5
        W = np.random.default_rng(r).standard_normal((8192, r)).astype(np.float32)
        ot.set_weights(W.astype(np.float64))
        Uo = ot.evaluate()
        gt.set_weights(torch.from_numpy(W).cuda())
        ref = None
        for sched in ("lpt", "tree_order"):
            for stages in (2, 3, 4):
                for runs in (False, True):
                    gt.set_launch(sched, stages, runs, False)
                    U = gt.evaluate().cpu().numpy()
                    assert np.linalg.norm(U - Uo) / np.linalg.norm(Uo) <= tol
                    if ref is None:
                        ref = U
                    assert np.array_equal(U, ref)
        for stages in (2, 3, 4):
            for runs in (False, True):
                gt.set_launch("lpt", stages, runs, True)
                U = gt.evaluate().cpu().numpy()
                assert np.linalg.norm(U - Uo) / np.linalg.norm(Uo) <= tol
                assert np.linalg.norm(U - ref) / np.linalg.norm(ref) <= 1e-6
    gt.close()


def test_autotune_needs_weights():
    from paper_1410_0260_gb300 import askit
    t = askit.Tree(torch.randn((2048, 8), device="cuda"), askit.Config(leaf_size=128, kappa=8, s_max=16))
    with pytest.raises(askit.AskitError):
        t.autotune()
    t.close()


def test_wide_kernel_schedules_match_the_oracle():
    """d = 100 (rows padded to 128: four K chunks of 32, the last partly
    outside the rows): both schedules and paired items, r = 1 and 3, against
    the oracle; the autotuner offers the paired items as a third candidate."""
    import oracle
    from paper_1410_0260_gb300 import askit, workloads
    X = workloads.mixture(3000, 100, 4, 3.0, seed=31)
    kw = dict(leaf_size=256, kappa=12, knn_mode=0, s_max=160, id_tol=1e-5, h=5.0, seed=9)
    ot = oracle.Tree(X, oracle.Config(**kw))
    gt = askit.Tree(torch.from_numpy(X).cuda(), askit.Config(precision="fp16x3", **kw))
    for r in (1, 3):
        W = np.random.default_rng(10 + r).standard_normal((3000, r)).astype(np.float32)
        ot.set_weights(W.astype(np.float64))
        Uo = ot.evaluate()
        gt.set_weights(torch.from_numpy(W).cuda())
        outs = []
        for sched in ("lpt", "tree_order"):
            gt.set_launch(sched, 3, True, False)
            U = gt.evaluate().cpu().numpy()
            assert np.linalg.norm(U - Uo) / np.linalg.norm(Uo) <= 1e-4, sched
            outs.append(U)
        assert np.array_equal(outs[0], outs[1])
        # paired 256-column items: each target row copied and split once for
        # both sub-blocks of a node; the sums differ by FP32 rounding only
        gt.set_launch("lpt", 3, True, True)
        U = gt.evaluate().cpu().numpy()
        assert np.linalg.norm(U - Uo) / np.linalg.norm(Uo) <= 1e-4
        assert np.linalg.norm(U - outs[0]) / np.linalg.norm(outs[0]) <= 1e-6
        gt.set_launch("lpt", 3, True, False)
    cands = gt.autotune(reps=1)
    assert len(cands) == 3 and sum(c["pairs"] for c in cands) == 1
    assert sum(c["chosen"] for c in cands) == 1
    gt.close()
