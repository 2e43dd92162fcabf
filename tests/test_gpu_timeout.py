"""The bounded waits of the FP16x3 evaluation kernels give up cleanly.

A tiny poll limit (askit_set_wait_limit) makes the kernel's mbarrier waits
run out on purpose.  The kernel must record the timeout (askit_sync reports
ASKIT_ERR_TIMEOUT once), leave every role's loop, wait for its copies and
MMAs in flight, free TMEM and return, so that the context stays usable: the
next evaluation with the default limit must match the oracle.  No GPU fault
is involved: the waits end by their own limit.
"""
import numpy as np
import pytest

import oracle
from paper_1410_0260_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_waits_give_up_and_the_tree_stays_usable():
    from paper_1410_0260_gb300 import askit
    w = wl.MANIFOLD_1M_64.scaled(16384)
    X, W = w.make_points(), w.make_weights()
    kw = dict(leaf_size=512, kappa=32, knn_mode=1, rp_iters=2, s_max=256, id_tol=1e-4, h=0.35, seed=2)
    otree = oracle.Tree(X, oracle.Config(**kw))
    otree.set_weights(W.astype(np.float64))
    Uo = otree.evaluate()
    t = askit.Tree(torch.from_numpy(X).cuda(), askit.Config(precision="fp16x3", **kw))
    t.set_weights(torch.from_numpy(W).cuda())
    for mode in ("global", "block"):
        t.set_fp16_centering(mode)
        for pairs in (False, True):
            t.set_launch("lpt", 2, True, pairs=pairs)
            t.set_wait_limit(1)
            t.evaluate()
            with pytest.raises(askit.AskitError, match="timed out"):
                t.sync()
            t.sync()                                   # reported once, then cleared
            t.set_wait_limit(0)
            U = t.evaluate().cpu().numpy()
            t.sync()
            err = float(np.linalg.norm(U - Uo) / np.linalg.norm(Uo))
            assert err <= (1e-4 if mode == "global" else 1e-5), (mode, pairs, err)
    t.close()
