"""The allocation-free exact kNN (askit_knn_noalloc), called through the C ABI.

Some callers cannot call cudaMalloc -- a serving process that reserved its
device memory up front, or a latency-critical caller that cannot take the
allocator's implicit synchronization -- so this entry point keeps its
scratch in a fixed device array inside the library.  It must return exactly
what the setup's exact kNN returns (ids and FP64 distances are bit-exact:
they are index work decided by the same FP64 arithmetic), on two calls in a
row (the array keeps the previous call's contents), and it must refuse
requests larger than its array.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_1410_0260_gb300 import askit
    return askit, askit.load()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_knn_noalloc_matches_setup_knn_on_two_calls():
    askit, L = _lib()
    from paper_1410_0260_gb300 import workloads
    X = workloads.mixture(3001, 7, 4, 5.0, seed=21)
    N, d, kappa = X.shape[0], X.shape[1], 16
    Xd = torch.from_numpy(X).cuda()
    tree = askit.Tree(Xd, askit.Config(leaf_size=128, kappa=kappa, knn_mode=0, s_max=16, precision="simt_fp32"))
    ref_ids = tree.structure(askit.STRUCT_KNN)
    ref_d = tree.structure(askit.STRUCT_KNN_DIST)
    for call in range(2):
        ids = torch.full((N, kappa), -7, dtype=torch.int32, device="cuda")
        dist = torch.full((N, kappa), -1.0, dtype=torch.float64, device="cuda")
        rc = L.askit_knn_noalloc(ctypes.c_void_p(Xd.data_ptr()), N, d, None, N, kappa,
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), _stream())
        assert rc == 0, L.askit_last_error()
        torch.cuda.synchronize()
        assert np.array_equal(ids.cpu().numpy(), ref_ids), call
        assert np.array_equal(dist.cpu().numpy(), ref_d), call
    tree.close()


def test_knn_noalloc_queries_and_limits():
    askit, L = _lib()
    rng = np.random.default_rng(5)
    X = rng.standard_normal((500, 5)).astype(np.float32)
    Y = rng.standard_normal((40, 5)).astype(np.float32)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    outs = []
    for call in range(2):
        ids = torch.zeros((40, 8), dtype=torch.int32, device="cuda")
        dist = torch.zeros((40, 8), dtype=torch.float64, device="cuda")
        rc = L.askit_knn_noalloc(ctypes.c_void_p(Xd.data_ptr()), 500, 5, ctypes.c_void_p(Yd.data_ptr()), 40, 8,
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), _stream())
        assert rc == 0, L.askit_last_error()
        torch.cuda.synchronize()
        outs.append((ids.cpu().numpy(), dist.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    # the nearest-first order and the reported distances hold up against float64 numpy
    D = ((Y[:, None, :].astype(np.float64) - X[None].astype(np.float64)) ** 2).sum(-1)
    assert np.allclose(outs[0][1], np.take_along_axis(D, outs[0][0].astype(np.int64), 1), rtol=1e-12)
    assert (np.diff(outs[0][1], axis=1) >= 0).all()
    # more queries than the scratch array holds: a clean error, no device work
    big = torch.zeros((8193, 5), dtype=torch.float32, device="cuda")
    ids = torch.zeros((8193, 8), dtype=torch.int32, device="cuda")
    dist = torch.zeros((8193, 8), dtype=torch.float64, device="cuda")
    rc = L.askit_knn_noalloc(ctypes.c_void_p(Xd.data_ptr()), 500, 5, ctypes.c_void_p(big.data_ptr()), 8193, 8,
                             ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), _stream())
    assert rc == 1 and b"at most 8192" in L.askit_last_error()
