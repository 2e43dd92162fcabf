"""Python binding of libaskit.so (the C ABI in include/askit.h).

Argument marshalling only: PyTorch supplies device memory and the stream;
every step of setup and evaluation runs in the library's CUDA kernels.  There
is no CPU path: if the shared library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass, field

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libaskit.so")
_lock = threading.Lock()
_lib = None

PREC_SIMT_FP32, PREC_TF32X3, PREC_BF16X3, PREC_FP16X3 = 0, 1, 2, 3
PRECISIONS = {"simt_fp32": PREC_SIMT_FP32, "tf32x3": PREC_TF32X3, "bf16x3": PREC_BF16X3, "fp16x3": PREC_FP16X3}
BW_CONSTANT, BW_ARRAY, BW_KNN = 0, 1, 2
(STRUCT_PERM, STRUCT_KNN, STRUCT_KNN_DIST, STRUCT_SKEL_S, STRUCT_SKEL_IDS, STRUCT_NL_CNT,
 STRUCT_NL_IDS, STRUCT_TROWS, STRUCT_HSRC, STRUCT_P, STRUCT_NCOL, STRUCT_WSKEL) = range(12)

EXPORTS = ["askit_default_params", "askit_setup", "askit_set_weights", "askit_evaluate",
           "askit_evaluate_targets", "askit_evaluate_host", "askit_set_precision", "askit_get_info",
           "askit_get_structure", "askit_sync", "askit_destroy", "askit_status_string",
           "askit_last_error", "askit_knn_noalloc", "askit_direct", "askit_weights_create",
           "askit_weights_set", "askit_weights_evaluate", "askit_weights_evaluate_targets",
           "askit_weights_destroy", "askit_footprint", "askit_graph_create", "askit_graph_launch",
           "askit_graph_destroy", "askit_autotune", "askit_set_launch", "askit_knn_targets",
           "askit_kernel_timing", "askit_set_wait_limit", "askit_set_fp16_centering", "askit_knn_points",
           "askit_evaluate_part", "askit_set_pruning", "askit_prune_stats"]


class TuneEntry(C.Structure):
    _fields_ = [("schedule", C.c_int32), ("stages", C.c_int32), ("tiled_runs", C.c_int32), ("pairs", C.c_int32),
                ("chosen", C.c_int32), ("ms", C.c_double)]


class AskitError(RuntimeError):
    pass


class Params(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("kappa", C.c_int32), ("knn_mode", C.c_int32),
                ("rp_iters", C.c_int32), ("rp_leaf", C.c_int32), ("s_max", C.c_int32),
                ("s_min", C.c_int32), ("ell_extra", C.c_int32), ("prune", C.c_int32),
                ("bw_mode", C.c_int32), ("bw_k", C.c_int32), ("precision", C.c_int32),
                ("id_tol", C.c_double), ("kernel_scale", C.c_double), ("h", C.c_double),
                ("seed", C.c_uint64), ("batch_entries", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("N", C.c_int64), ("d", C.c_int32), ("d_pad", C.c_int32), ("L", C.c_int32),
                ("kappa", C.c_int32), ("r", C.c_int32), ("n_nodes", C.c_int64),
                ("skel_total", C.c_int64), ("skel_rows_padded", C.c_int64), ("n_blocks", C.c_int64),
                ("n_items", C.c_int64), ("n_entries", C.c_int64), ("pairs_algorithmic", C.c_int64), ("pairs_computed", C.c_int64),
                ("near_total", C.c_int64), ("far_total", C.c_int64), ("device_bytes", C.c_int64),
                ("n_batches", C.c_int64), ("setup_ms", C.c_double * 7), ("fp16_centering", C.c_int32),
                ("pad_", C.c_int32), ("fp16_rho", C.c_double)]


def prune_stats(X: torch.Tensor, leaf_size: int, kappa: int, rscale: float = 1.0, stream=None):
    """Nodes visited per target under neighbor and distance pruning (Section
    3, Table 1): (visited_knn [N], visited_dist [N]) int64 on X's device."""
    X = _dev_f32(X, "X")
    N, d = X.shape
    vk = torch.empty(N, dtype=torch.int64, device=X.device)
    vd = torch.empty(N, dtype=torch.int64, device=X.device)
    _check(load().askit_prune_stats(C.c_void_p(X.data_ptr()), N, d, X.stride(0), leaf_size, kappa, float(rscale),
                                    C.c_void_p(vk.data_ptr()), C.c_void_p(vd.data_ptr()), _stream(stream)))
    return vk, vd


def load(path: str | None = None):
    """Load libaskit.so (built by build.py / __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            p = path or LIB_PATH
            if not os.path.exists(p):
                raise AskitError(f"libaskit.so not built ({p}); run __graft_entry__.build()")
            L = C.CDLL(p)
            V, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
            L.askit_default_params.argtypes = [C.POINTER(Params)]
            L.askit_setup.argtypes = [V, I64, I32, I64, V, V, C.POINTER(Params), V, C.POINTER(V)]
            L.askit_set_weights.argtypes = [V, V, I32, I64, V]
            L.askit_evaluate.argtypes = [V, V, I64, V]
            L.askit_evaluate_targets.argtypes = [V, V, I64, I64, V, I64, V]
            L.askit_evaluate_host.argtypes = [V, V, I32, I64, V, I64, V]
            L.askit_set_precision.argtypes = [V, I32]
            L.askit_get_info.argtypes = [V, C.POINTER(Info)]
            L.askit_get_structure.argtypes = [V, I32, V, C.c_size_t]
            L.askit_sync.argtypes = [V, V]
            L.askit_destroy.argtypes = [V]
            L.askit_knn_noalloc.argtypes = [V, I64, I32, V, I64, I32, V, V, V]
            L.askit_direct.argtypes = [V, V, I64, V, I64, V]
            L.askit_weights_create.argtypes = [V, C.POINTER(V)]
            L.askit_weights_set.argtypes = [V, V, I32, I64, V]
            L.askit_weights_evaluate.argtypes = [V, V, I64, V]
            L.askit_weights_evaluate_targets.argtypes = [V, V, I64, I64, V, I64, V]
            L.askit_weights_destroy.argtypes = [V]
            L.askit_footprint.argtypes = [V, I32, I64, I32, C.POINTER(C.c_size_t)]
            L.askit_graph_create.argtypes = [V, V, I32, I64, V, I64, V, C.POINTER(V)]
            L.askit_graph_launch.argtypes = [V, V]
            L.askit_graph_destroy.argtypes = [V]
            L.askit_autotune.argtypes = [V, I32, V, C.POINTER(TuneEntry), I32, C.POINTER(I32)]
            L.askit_set_launch.argtypes = [V, I32, I32, I32, I32]
            L.askit_set_wait_limit.argtypes = [V, I32]
            L.askit_set_fp16_centering.argtypes = [V, I32]
            L.askit_knn_points.argtypes = [V, V, I64, V, V, V]
            L.askit_evaluate_part.argtypes = [V, I32, V, I64, V]
            L.askit_set_pruning.argtypes = [V, I32, D, V]
            L.askit_prune_stats.argtypes = [V, I64, I32, I64, I32, I32, D, V, V, V]
            L.askit_knn_targets.argtypes = [V, V, I64, I64, V, V, V]
            L.askit_kernel_timing.argtypes = [V, I32, C.POINTER(D), C.POINTER(I64)]
            L.askit_status_string.restype = C.c_char_p
            L.askit_status_string.argtypes = [C.c_int]
            L.askit_last_error.restype = C.c_char_p
            for name in EXPORTS:
                if name not in ("askit_status_string", "askit_last_error", "askit_default_params"):
                    getattr(L, name).restype = C.c_int
            _lib = L
    return _lib


def _check(rc: int):
    if rc != 0:
        L = load()
        raise AskitError(f"{L.askit_status_string(rc).decode()}: {L.askit_last_error().decode()}")


def _stream(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _dev_f32(a: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(a, torch.Tensor) and a.is_cuda and a.dtype == torch.float32):
        raise AskitError(f"{name} must be a CUDA float32 tensor")
    if a.dim() == 1:
        a = a.view(-1, 1)
    if a.stride(1) != 1:
        a = a.contiguous()
    return a


@dataclass
class Config:
    """ASKIT parameters (Section 3: m, kappa, s, ell; Section 4: h)."""
    leaf_size: int = 128
    kappa: int = 16
    knn_mode: int = 0
    rp_iters: int = 4
    rp_leaf: int = 0
    s_max: int = 64
    s_min: int = 1
    ell_extra: int = 20
    prune: int = 1              # 1 eq. (2.5) per target, 0 none, 2 leaf-grouped lists
    bw_mode: int = BW_CONSTANT
    bw_k: int = 16
    precision: str = "tf32x3"
    id_tol: float = 1e-6
    kernel_scale: float = 0.5
    h: float = 1.0
    seed: int = 1
    batch_entries: int = 0      # entries per in-sample work-list batch (0 = 2^28)

    def to_c(self) -> Params:
        return Params(self.leaf_size, self.kappa, self.knn_mode, self.rp_iters, self.rp_leaf, self.s_max,
                      self.s_min, self.ell_extra, self.prune, self.bw_mode, self.bw_k,
                      PRECISIONS[self.precision], self.id_tol, self.kernel_scale, self.h, self.seed,
                      self.batch_entries)


class Tree:
    """A skeletonized ASKIT tree resident on the GPU."""

    def __init__(self, X: torch.Tensor, cfg: Config, h: torch.Tensor | None = None,
                 knn: torch.Tensor | None = None, stream=None):
        L = load()
        X = _dev_f32(X, "X")
        self.N, self.d = X.shape
        self.cfg = cfg
        self.device = X.device
        p = cfg.to_c()
        hp = None
        if h is not None:
            h = _dev_f32(h, "h").contiguous()
            hp = C.c_void_p(h.data_ptr())
        kp = None
        if knn is not None:
            knn = knn.to(device=X.device, dtype=torch.int32).contiguous()
            kp = C.c_void_p(knn.data_ptr())
        out = C.c_void_p()
        with torch.cuda.device(X.device):
            _check(L.askit_setup(C.c_void_p(X.data_ptr()), self.N, self.d, X.stride(0), hp, kp,
                                 C.byref(p), _stream(stream), C.byref(out)))
        self._t = out
        self.r = 0
        self.kappa = cfg.kappa

    def close(self):
        if getattr(self, "_t", None):
            load().askit_destroy(self._t)
            self._t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ calls
    def set_precision(self, precision: str):
        _check(load().askit_set_precision(self._t, PRECISIONS[precision]))

    def set_weights(self, W: torch.Tensor, stream=None):
        W = _dev_f32(W, "W")
        _check(load().askit_set_weights(self._t, C.c_void_p(W.data_ptr()), W.shape[1], W.stride(0),
                                        _stream(stream)))
        self._W = W   # keep alive until the stream has consumed it
        self.r = W.shape[1]

    def evaluate(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.N, max(self.r, 1)), dtype=torch.float32, device=self.device)
        out = _dev_f32(out, "out")
        _check(load().askit_evaluate(self._t, C.c_void_p(out.data_ptr()), out.stride(0), _stream(stream)))
        return out

    def evaluate_targets(self, Y: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        Y = _dev_f32(Y, "Y")
        if out is None:
            out = torch.empty((Y.shape[0], max(self.r, 1)), dtype=torch.float32, device=self.device)
        _check(load().askit_evaluate_targets(self._t, C.c_void_p(Y.data_ptr()), Y.shape[0], Y.stride(0),
                                             C.c_void_p(out.data_ptr()), out.stride(0), _stream(stream)))
        return out

    def evaluate_host(self, W: np.ndarray, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        W = np.ascontiguousarray(W, dtype=np.float32).reshape(self.N, -1)
        r = W.shape[1]
        if out is None:
            out = np.empty((self.N, r), np.float32)
        _check(load().askit_evaluate_host(self._t, W.ctypes.data_as(C.c_void_p), r, r,
                                          out.ctypes.data_as(C.c_void_p), out.shape[1], _stream(stream)))
        self.r = r
        return out

    def evaluate_host_ptr(self, W_ptr: int, r: int, U_ptr: int, stream=None):
        """End-to-end call on caller-owned (e.g. pinned) host buffers."""
        _check(load().askit_evaluate_host(self._t, C.c_void_p(W_ptr), r, r, C.c_void_p(U_ptr), r,
                                          _stream(stream)))
        self.r = r

    def knn_targets(self, Y: torch.Tensor, stream=None) -> tuple[torch.Tensor, torch.Tensor]:
        """Exact kappa nearest tree points of each row of Y: (ids, squared distances)."""
        Y = _dev_f32(Y, "Y")
        kappa = self.info()["kappa"]
        ids = torch.empty((Y.shape[0], kappa), dtype=torch.int32, device=self.device)
        dist = torch.empty((Y.shape[0], kappa), dtype=torch.float64, device=self.device)
        _check(load().askit_knn_targets(self._t, C.c_void_p(Y.data_ptr()), Y.shape[0], Y.stride(0),
                                        C.c_void_p(ids.data_ptr()), C.c_void_p(dist.data_ptr()), _stream(stream)))
        return ids, dist

    def direct(self, targets, stream=None) -> torch.Tensor:
        """Exact direct sum (eq. 1.1) at the given point ids, with the current weights."""
        tg = torch.as_tensor(targets, dtype=torch.int32, device=self.device).contiguous()
        out = torch.empty((tg.numel(), max(self.r, 1)), dtype=torch.float32, device=self.device)
        _check(load().askit_direct(self._t, C.c_void_p(tg.data_ptr()), tg.numel(), C.c_void_p(out.data_ptr()),
                                   out.stride(0), _stream(stream)))
        return out

    def knn_points(self, ids, stream=None):
        """Exact kappa nearest neighbors of the tree's points `ids` (self
        excluded): (ids [Q, kappa] int32, squared distances [Q, kappa] FP64)."""
        q = torch.as_tensor(ids, dtype=torch.int32, device=self.device).contiguous()
        nb = torch.empty((q.numel(), self.kappa), dtype=torch.int32, device=self.device)
        dd = torch.empty((q.numel(), self.kappa), dtype=torch.float64, device=self.device)
        _check(load().askit_knn_points(self._t, C.c_void_p(q.data_ptr()), q.numel(), C.c_void_p(nb.data_ptr()),
                                       C.c_void_p(dd.data_ptr()), _stream(stream)))
        return nb, dd

    def evaluate_part(self, part: str, U: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Evaluate with the near field only ("near") or the far field only ("far")."""
        if U is None:
            U = torch.empty((self.N, max(self.r, 1)), dtype=torch.float32, device=self.device)
        _check(load().askit_evaluate_part(self._t, {"all": 0, "near": 1, "far": 2}[part], C.c_void_p(U.data_ptr()),
                                          U.stride(0), _stream(stream)))
        return U

    def sync(self, stream=None):
        _check(load().askit_sync(self._t, _stream(stream)))

    def weights_context(self) -> "Weights":
        return Weights(self)

    def autotune(self, reps: int = 3, stream=None) -> list[dict]:
        """Time the evaluation kernel's launch configurations on this tree
        (weights must be set) and keep the fastest; returns every candidate."""
        out = (TuneEntry * 32)()
        n = C.c_int32()
        _check(load().askit_autotune(self._t, reps, _stream(stream), out, 32, C.byref(n)))
        return [{"schedule": ("lpt", "tree_order", "lpt_pairs")[e.schedule], "stages": e.stages,
                 "tiled_runs": bool(e.tiled_runs), "pairs": bool(e.pairs), "chosen": bool(e.chosen), "ms": e.ms}
                for e in out[:n.value]]

    def set_launch(self, schedule: str = "lpt", stages: int = 3, tiled_runs: bool = True, pairs: bool = False):
        """Set the evaluation kernel's launch configuration (see autotune)."""
        _check(load().askit_set_launch(self._t, {"lpt": 0, "tree_order": 1}[schedule], stages, int(tiled_runs),
                                       int(pairs)))

    def set_pruning(self, far_height: int = -1, kappa_cut: float = 0.0, stream=None):
        """Level-restricted far field (far_height >= 0) and adaptive kappa_i
        (kappa_cut > 0); rebuilds the work lists.  Weights stay valid unless
        the lists outgrow a weight context's partial sums: its evaluations
        then raise NOT_READY until its weights are set again."""
        _check(load().askit_set_pruning(self._t, int(far_height), float(kappa_cut), _stream(stream)))

    def set_fp16_centering(self, mode: str = "auto"):
        """FP16x3 target centering: "auto", "block" (per source sub-block, on
        the chip) or "global" (pre-split around the data mean)."""
        _check(load().askit_set_fp16_centering(self._t, {"auto": 0, "block": 1, "global": 2}[mode]))

    def set_wait_limit(self, polls: int):
        """Poll limit of the FP16x3 kernel's bounded waits (0: the default);
        a debugging and test aid -- a tiny limit makes the waits give up."""
        _check(load().askit_set_wait_limit(self._t, int(polls)))

    def kernel_timing(self, enable: bool):
        """Start (True) or end (False) timing the evaluation kernel's own
        launches with CUDA events; ending returns (total ms, launches)."""
        ms, n = C.c_double(), C.c_int64()
        _check(load().askit_kernel_timing(self._t, int(enable), C.byref(ms), C.byref(n)))
        return None if enable else (ms.value, n.value)

    def capture(self, W: torch.Tensor, U: torch.Tensor, stream=None) -> "Graph":
        """A CUDA graph of set_weights(W) + evaluate(U); replays read W's
        current contents and overwrite U."""
        return Graph(self, W, U, stream)

    def footprint(self, kind: int, n: int, r: int) -> int:
        b = C.c_size_t()
        _check(load().askit_footprint(self._t, kind, n, r, C.byref(b)))
        return b.value

    def info(self) -> dict:
        inf = Info()
        _check(load().askit_get_info(self._t, C.byref(inf)))
        out = {k: getattr(inf, k) for k, _ in Info._fields_}
        out["setup_ms"] = dict(zip(("knn", "tree", "node_lists", "sampling", "skeletons", "operands", "work_lists"),
                                   list(inf.setup_ms)))
        return out

    def structure(self, which: int) -> np.ndarray:
        inf = self.info()
        N, kappa, nn = inf["N"], inf["kappa"], inf["n_nodes"]
        ell = self.cfg.s_max + self.cfg.ell_extra
        shapes = {STRUCT_PERM: ((N,), np.int32), STRUCT_KNN: ((N, kappa), np.int32),
                  STRUCT_KNN_DIST: ((N, kappa), np.float64), STRUCT_SKEL_S: ((nn,), np.int32),
                  STRUCT_SKEL_IDS: ((inf["skel_total"],), np.int32), STRUCT_NL_CNT: ((nn,), np.int32),
                  STRUCT_NL_IDS: ((nn, ell), np.int32), STRUCT_TROWS: ((nn, ell), np.int32),
                  STRUCT_HSRC: ((N,), np.float32), STRUCT_NCOL: ((nn,), np.int32),
                  STRUCT_WSKEL: ((inf["skel_total"], max(inf["r"], 1)), np.float32)}
        if which == STRUCT_P:
            s = self.structure(STRUCT_SKEL_S).astype(np.int64)
            c = self.structure(STRUCT_NCOL).astype(np.int64)
            shape, dt = ((int((s * (c - s)).sum()),), np.float64)
        else:
            shape, dt = shapes[which]
        a = np.zeros(shape, dt)
        _check(load().askit_get_structure(self._t, which, a.ctypes.data_as(C.c_void_p), a.nbytes))
        return a


class Weights:
    """A weight context of a tree (independent of the tree's default weights)."""

    def __init__(self, tree: Tree):
        self.tree = tree
        h = C.c_void_p()
        _check(load().askit_weights_create(tree._t, C.byref(h)))
        self._w = h
        self.r = 0

    def set(self, W: torch.Tensor, stream=None):
        W = _dev_f32(W, "W")
        _check(load().askit_weights_set(self._w, C.c_void_p(W.data_ptr()), W.shape[1], W.stride(0), _stream(stream)))
        self._W = W
        self.r = W.shape[1]

    def evaluate(self, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.tree.N, max(self.r, 1)), dtype=torch.float32, device=self.tree.device)
        _check(load().askit_weights_evaluate(self._w, C.c_void_p(out.data_ptr()), out.stride(0), _stream(stream)))
        return out

    def evaluate_targets(self, Y: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        Y = _dev_f32(Y, "Y")
        if out is None:
            out = torch.empty((Y.shape[0], max(self.r, 1)), dtype=torch.float32, device=self.tree.device)
        _check(load().askit_weights_evaluate_targets(self._w, C.c_void_p(Y.data_ptr()), Y.shape[0], Y.stride(0),
                                                     C.c_void_p(out.data_ptr()), out.stride(0), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_w", None):
            load().askit_weights_destroy(self._w)
            self._w = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """A captured weights + Evaluate step (askit_graph_*)."""

    def __init__(self, tree: Tree, W: torch.Tensor, U: torch.Tensor, stream=None):
        # the graph binds these buffers' addresses: no copies here
        for name, a in (("W", W), ("U", U)):
            if not (a.is_cuda and a.dtype == torch.float32 and a.dim() == 2 and a.stride(1) == 1):
                raise AskitError(f"{name} must be a row-major 2-D FP32 CUDA tensor")
        if W.shape[0] != tree.N or U.shape != W.shape:
            raise AskitError("W and U must both be [N, r]")
        self.tree, self.W, self.U = tree, W, U
        h = C.c_void_p()
        _check(load().askit_graph_create(tree._t, C.c_void_p(W.data_ptr()), W.shape[1], W.stride(0),
                                         C.c_void_p(U.data_ptr()), U.stride(0), _stream(stream), C.byref(h)))
        self._g = h

    def launch(self, stream=None):
        _check(load().askit_graph_launch(self._g, _stream(stream)))

    def close(self):
        if getattr(self, "_g", None):
            load().askit_graph_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
