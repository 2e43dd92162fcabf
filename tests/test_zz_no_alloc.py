"""The allocation-free exact kNN (askit_knn_noalloc), called through the C ABI.

Some callers cannot call cudaMalloc -- a serving process that reserved its
device memory up front, or a latency-critical caller that cannot take the
allocator's implicit synchronization -- so this entry point keeps its
scratch in a fixed device array inside the library.  Its lists must be the
exact kNN as the FP64 oracle defines it (ids and FP64 distances bit-exact:
index work decided by the same canonical FP64 arithmetic, ties by id), on
two calls in a row (the array keeps the previous call's contents); it must
take no device memory, and it must refuse requests larger than its array.
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    from paper_1410_0260_gb300 import askit
    return askit, askit.load()


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _call(L, Xd, N, d, Yd, Q, kappa):
    ids = torch.full((Q, kappa), -7, dtype=torch.int32, device="cuda")
    dist = torch.full((Q, kappa), -1.0, dtype=torch.float64, device="cuda")
    rc = L.askit_knn_noalloc(ctypes.c_void_p(Xd.data_ptr()), N, d,
                             None if Yd is None else ctypes.c_void_p(Yd.data_ptr()), Q, kappa,
                             ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), _stream())
    assert rc == 0, L.askit_last_error()
    torch.cuda.synchronize()
    return ids, dist


def test_knn_noalloc_matches_the_oracle_on_two_calls():
    askit, L = _lib()
    from paper_1410_0260_gb300 import workloads
    X = workloads.mixture(3001, 7, 4, 5.0, seed=21)
    N, d, kappa = X.shape[0], X.shape[1], 16
    ref_ids, ref_d = oracle.knn_exact(X, kappa)
    Xd = torch.from_numpy(X).cuda()
    for call in range(2):
        ids, dist = _call(L, Xd, N, d, None, N, kappa)
        assert np.array_equal(ids.cpu().numpy(), ref_ids), call
        assert np.array_equal(dist.cpu().numpy(), ref_d), call


def test_knn_noalloc_queries_with_ties_and_limits():
    askit, L = _lib()
    rng = np.random.default_rng(5)
    X = rng.standard_normal((500, 5)).astype(np.float32)
    X[250:300] = X[200:250]                       # duplicated points: ties broken by id
    Y = np.concatenate([rng.standard_normal((30, 5)).astype(np.float32), X[195:205]])
    ref_ids, ref_d = oracle.knn_exact(X, 8, Y=Y)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    for call in range(2):
        ids, dist = _call(L, Xd, 500, 5, Yd, Y.shape[0], 8)
        assert np.array_equal(ids.cpu().numpy(), ref_ids), call
        assert np.array_equal(dist.cpu().numpy(), ref_d), call
    # more queries than the scratch array holds: a clean error, no device work
    big = torch.zeros((8193, 5), dtype=torch.float32, device="cuda")
    ids = torch.zeros((8193, 8), dtype=torch.int32, device="cuda")
    dist = torch.zeros((8193, 8), dtype=torch.float64, device="cuda")
    rc = L.askit_knn_noalloc(ctypes.c_void_p(Xd.data_ptr()), 500, 5, ctypes.c_void_p(big.data_ptr()), 8193, 8,
                             ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), _stream())
    assert rc == 1 and b"at most 8192" in L.askit_last_error()


def test_knn_noalloc_takes_no_device_memory():
    askit, L = _lib()
    rng = np.random.default_rng(8)
    X = rng.standard_normal((4000, 12)).astype(np.float32)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(rng.standard_normal((700, 12)).astype(np.float32)).cuda()
    ids = torch.zeros((700, 32), dtype=torch.int32, device="cuda")
    dist = torch.zeros((700, 32), dtype=torch.float64, device="cuda")

    def call():
        rc = L.askit_knn_noalloc(ctypes.c_void_p(Xd.data_ptr()), 4000, 12, ctypes.c_void_p(Yd.data_ptr()), 700, 32,
                                 ctypes.c_void_p(ids.data_ptr()), ctypes.c_void_p(dist.data_ptr()), _stream())
        assert rc == 0, L.askit_last_error()

    call()                                        # the first call looks up the array's address
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
