"""ASKIT oracle: plain, slow, FP64 CPU restatement of the paper's method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
library (``paper_1410_0260_gb300``) never imports, links or executes it, and
the two share no code: the oracle is C compiled by gcc (``askit_oracle.c``),
the product path is CUDA.

This module only marshals numpy arrays into the C functions; all arithmetic
lives in ``askit_oracle.c`` with a citation at every function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "askit_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liborc.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # ASKIT_ORACLE_LIB loads a separately built copy (used to check that
            # planted mistakes in the oracle are caught by its pins)
            _lib = C.CDLL(os.environ.get("ASKIT_ORACLE_LIB") or build())
            _declare(_lib)
    return _lib


P = C.c_void_p
i64 = C.c_int64
i32 = C.c_int


class Params(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("kappa", C.c_int32), ("knn_mode", C.c_int32),
                ("rp_iters", C.c_int32), ("rp_leaf", C.c_int32), ("s_max", C.c_int32),
                ("s_min", C.c_int32), ("ell_extra", C.c_int32), ("prune", C.c_int32),
                ("bw_mode", C.c_int32), ("bw_k", C.c_int32), ("pad_", C.c_int32),
                ("id_tol", C.c_double), ("kscale", C.c_double), ("h", C.c_double),
                ("seed", C.c_uint64)]


def _declare(L):
    L.orc_philox4x64_10.argtypes = [P, P, P]
    L.orc_cexp.argtypes = [C.c_double]
    L.orc_cexp.restype = C.c_double
    L.orc_direct.argtypes = [P, i64, i32, P, C.c_double, P, i32, P, P, i64, P]
    L.orc_knn_exact.argtypes = [P, i64, i32, i32, P, P, i64, P, P]
    L.orc_knn_rp.argtypes = [P, i64, i32, i32, i32, i64, C.c_uint64, P, P]
    L.orc_tree_depth.argtypes = [i64, i64]
    L.orc_tree_depth.restype = i32
    L.orc_askit_tree.argtypes = [P, i64, i32, i64, P]
    L.orc_askit_tree.restype = i32
    L.orc_cpqr_id.argtypes = [P, i32, i32, C.c_double, i32, i32, P, P, P]
    L.orc_cpqr_id.restype = i32
    L.orc_build.argtypes = [P, i64, i32, C.POINTER(Params), P, P]
    L.orc_build.restype = P
    L.orc_set_weights.argtypes = [P, P, i32]
    L.orc_evaluate.argtypes = [P, P, i64, P, P, P]
    L.orc_evaluate_part.argtypes = [P, P, i64, i32, P, P, P]
    L.orc_prune_stats.argtypes = [P, i64, i32, i64, i32, C.c_double, P, P]
    L.orc_prune_stats.restype = i32
    L.orc_evaluate_ext.argtypes = [P, P, i64, i32, i32, C.c_double, P, P, P]
    L.orc_evaluate_oos_ext.argtypes = [P, P, i64, i32, C.c_double, P, P, P, P]
    L.orc_evaluate_oos.argtypes = [P, P, i64, P, P, P, P]
    L.orc_info.argtypes = [P, P]
    L.orc_get_perm.argtypes = [P, P]
    L.orc_get_knn.argtypes = [P, P, P]
    L.orc_get_hsrc.argtypes = [P, P]
    L.orc_get_counts.argtypes = [P, P, P, P, P, P, P]
    L.orc_get_node.argtypes = [P, i64, P, P, P, P, P, P, P, P]
    L.orc_free.argtypes = [P]
    L.orc_num_threads.restype = i32
    L.orc_set_threads.argtypes = [i32]


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops (results do not depend on it)."""
    lib().orc_set_threads(int(n))


def philox4x64_10(ctr, key):
    c = np.asarray(ctr, dtype=np.uint64)
    k = np.asarray(key, dtype=np.uint64)
    out = np.zeros(4, np.uint64)
    lib().orc_philox4x64_10(_p(c), _p(k), _p(out))
    return out


def cexp(a: float) -> float:
    return lib().orc_cexp(float(a))


def direct(X, W, h, kscale, targets=None, Y=None):
    """u = sum_j exp(-c ||x - x_j||^2 / h_j^2) w_j at points `targets` (ids) or at Y."""
    X = _f32(X)
    N, d = X.shape
    W = _f64(W).reshape(N, -1)
    r = W.shape[1]
    hs = _f32(np.broadcast_to(np.asarray(h, np.float32), (N,)))
    if Y is not None:
        Y = _f32(Y)
        T = Y.shape[0]
        tg = None
    else:
        tg = np.ascontiguousarray(targets, dtype=np.int64)
        T = tg.shape[0]
    U = np.zeros((T, r), np.float64)
    lib().orc_direct(_p(X), N, d, _p(hs), float(kscale), _p(W), r, _p(Y), _p(tg), T, _p(U))
    return U


def knn_exact(X, kappa, rows=None, Y=None):
    X = _f32(X)
    N, d = X.shape
    if Y is not None:
        Y = _f32(Y)
        Q = Y.shape[0]
        rw = None
    else:
        rw = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
        Q = rw.shape[0]
    ids = np.zeros((Q, kappa), np.int32)
    dd = np.zeros((Q, kappa), np.float64)
    lib().orc_knn_exact(_p(X), N, d, kappa, _p(Y), _p(rw), Q, _p(ids), _p(dd))
    return ids, dd


def knn_rp(X, kappa, iters, rp_leaf, seed):
    X = _f32(X)
    N, d = X.shape
    ids = np.zeros((N, kappa), np.int32)
    dd = np.zeros((N, kappa), np.float64)
    lib().orc_knn_rp(_p(X), N, d, kappa, iters, rp_leaf, seed, _p(ids), _p(dd))
    return ids, dd


def prune_stats(X, m, kappa, rscale=1.0):
    """Nodes the downward pass visits per target (Table 1 of Section 3)
    under neighbor pruning (exact kNN, kappa neighbors) and under distance
    pruning (centroid, radius R scaled by rscale): (L, visited_knn [N],
    visited_dist [N]); the tree has 2^(L+1) - 1 nodes."""
    X = _f32(X)
    N, d = X.shape
    vk = np.zeros(N, np.int64)
    vd = np.zeros(N, np.int64)
    L = lib().orc_prune_stats(_p(X), N, d, m, kappa, float(rscale), _p(vk), _p(vd))
    return L, vk, vd


def hit_rate(ids, ids_exact):
    """hr of Section 4: the mean fraction of the exact kappa nearest
    neighbors found in each approximate list (rows compared as sets)."""
    ids, ids_exact = np.asarray(ids), np.asarray(ids_exact)
    hits = [len(set(a.tolist()) & set(b.tolist())) for a, b in zip(ids, ids_exact)]
    return float(np.mean(hits)) / ids.shape[1]


def tree_depth(N, leaf):
    return lib().orc_tree_depth(N, leaf)


def askit_tree(X, m):
    X = _f32(X)
    N, d = X.shape
    perm = np.zeros(N, np.int64)
    L = lib().orc_askit_tree(_p(X), N, d, m, _p(perm))
    return perm, L


def cpqr_id(A, tol, s_lo, s_hi):
    """Pivoted-QR interpolative decomposition of A (rows x cols). Returns (piv, P, s, rdiag)."""
    A = _f64(A).copy()
    rows, cols = A.shape
    piv = np.zeros(cols, np.int32)
    Pm = np.zeros(max(1, min(s_hi, cols, rows) * cols), np.float64)
    rd = np.zeros(max(1, cols), np.float64)
    s = lib().orc_cpqr_id(_p(A), rows, cols, float(tol), s_lo, s_hi, _p(piv), _p(Pm), _p(rd))
    return piv, Pm[: s * (cols - s)].reshape(s, cols - s), s, rd[:s]


@dataclass
class Config:
    leaf_size: int
    kappa: int
    knn_mode: int = 0
    rp_iters: int = 4
    rp_leaf: int = 0
    s_max: int = 64
    s_min: int = 1
    ell_extra: int = 20
    prune: int = 1              # 0 none, 1 eq. (2.5) per target, 2 leaf-grouped lists
    bw_mode: int = 0
    bw_k: int = 16
    id_tol: float = 1e-6
    kscale: float = 0.5
    h: float = 1.0
    seed: int = 1

    def to_c(self) -> Params:
        rp_leaf = self.rp_leaf or max(2 * self.kappa + 2, self.leaf_size)
        return Params(self.leaf_size, self.kappa, self.knn_mode, self.rp_iters, rp_leaf,
                      self.s_max, self.s_min, self.ell_extra, self.prune, self.bw_mode,
                      self.bw_k, 0, self.id_tol, self.kscale, self.h, self.seed)


class Tree:
    """The oracle's full ASKIT structure (Algorithm 5 up to Evaluate)."""

    def __init__(self, X, cfg: Config, hsrc=None, knn=None):
        self.X = _f32(X)
        self.N, self.d = self.X.shape
        self.cfg = cfg
        self._prm = cfg.to_c()
        self._h = None if hsrc is None else _f32(hsrc)
        self._knn = None if knn is None else np.ascontiguousarray(knn, np.int32)
        self._t = lib().orc_build(_p(self.X), self.N, self.d, C.byref(self._prm),
                                  _p(self._h), _p(self._knn))
        info = np.zeros(8, np.int64)
        lib().orc_info(self._t, _p(info))
        self.L = int(info[2])
        self.nnodes = int(info[3])
        self.r = 0

    def __del__(self):
        t = getattr(self, "_t", None)
        if t:
            lib().orc_free(t)
            self._t = None

    # --- structure ---------------------------------------------------------
    def perm(self):
        p = np.zeros(self.N, np.int64)
        lib().orc_get_perm(self._t, _p(p))
        return p

    def knn(self):
        k = self.cfg.kappa
        ids = np.zeros((self.N, k), np.int32)
        dd = np.zeros((self.N, k), np.float64)
        lib().orc_get_knn(self._t, _p(ids), _p(dd))
        return ids, dd

    def hsrc(self):
        h = np.zeros(self.N, np.float32)
        lib().orc_get_hsrc(self._t, _p(h))
        return h

    def counts(self):
        arrs = [np.zeros(self.nnodes, np.int64) for _ in range(6)]
        lib().orc_get_counts(self._t, *[_p(a) for a in arrs])
        return dict(zip(["start", "size", "nl", "ell", "ncol", "s"], arrs))

    def node(self, a):
        c = self.counts()
        nl, ell, ncol, s = int(c["nl"][a]), int(c["ell"][a]), int(c["ncol"][a]), int(c["s"][a])
        out = dict(nl_ids=np.zeros(nl, np.int32), nl_key=np.zeros(nl, np.float64),
                   trows=np.zeros(ell, np.int32), cols=np.zeros(ncol, np.int32),
                   piv=np.zeros(ncol, np.int32), skel=np.zeros(s, np.int32),
                   P=np.zeros((s, ncol - s), np.float64), wsk=np.zeros((s, max(self.r, 1)), np.float64))
        lib().orc_get_node(self._t, a, *[_p(out[k]) for k in
                                         ["nl_ids", "nl_key", "trows", "cols", "piv", "skel", "P", "wsk"]])
        if self.r == 0:
            out["wsk"] = out["wsk"][:, :0]
        return out

    # --- weights and evaluation ---------------------------------------------
    def set_weights(self, W):
        W = _f64(W).reshape(self.N, -1)
        self.r = W.shape[1]
        self._W = W
        lib().orc_set_weights(self._t, _p(W), self.r)

    def evaluate(self, targets=None, counts=False):
        tg = np.arange(self.N, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        T = tg.shape[0]
        U = np.zeros((T, self.r), np.float64)
        near = np.zeros(T, np.int64)
        far = np.zeros(T, np.int64)
        lib().orc_evaluate(self._t, _p(tg), T, _p(U), _p(near), _p(far))
        return (U, near, far) if counts else U

    def evaluate_part(self, part, targets=None):
        """Algorithm 4 with only the near field ("near": direct leaf sums) or
        only the far field ("far": skeleton sums); near + far = evaluate()."""
        tg = np.arange(self.N, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        U = np.zeros((tg.shape[0], self.r), np.float64)
        lib().orc_evaluate_part(self._t, _p(tg), tg.shape[0], {"near": 1, "far": 2}[part], _p(U), None, None)
        return U

    def evaluate_ext(self, far_height=-1, kappa_cut=0.0, targets=None, counts=False, part="all"):
        """Algorithm 4 with the paper's proposed refinements (Section 3):
        far_height >= 0 uses skeletons only for nodes at most that many
        levels above the leaves; kappa_cut > 0 keeps in each prune set the
        neighbors up to the last one whose kernel value exceeds e^-kappa_cut."""
        tg = np.arange(self.N, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
        T = tg.shape[0]
        U = np.zeros((T, self.r), np.float64)
        near = np.zeros(T, np.int64)
        far = np.zeros(T, np.int64)
        lib().orc_evaluate_ext(self._t, _p(tg), T, {"near": 1, "far": 2, "all": 3}[part], int(far_height),
                               float(kappa_cut), _p(U), _p(near), _p(far))
        return (U, near, far) if counts else U

    def evaluate_oos_ext(self, Y, far_height=-1, kappa_cut=0.0):
        Y = _f32(Y)
        T = Y.shape[0]
        U = np.zeros((T, self.r), np.float64)
        lib().orc_evaluate_oos_ext(self._t, _p(Y), T, int(far_height), float(kappa_cut), _p(U), None, None, None)
        return U

    def evaluate_oos(self, Y, counts=False):
        Y = _f32(Y)
        T = Y.shape[0]
        U = np.zeros((T, self.r), np.float64)
        near = np.zeros(T, np.int64)
        far = np.zeros(T, np.int64)
        knn = np.zeros((T, self.cfg.kappa), np.int32)
        lib().orc_evaluate_oos(self._t, _p(Y), T, _p(U), _p(knn), _p(near), _p(far))
        return (U, knn, near, far) if counts else U
