"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws random numbers; it holds none of the method's
arithmetic, so both the CUDA path and the CPU oracle can consume its output.

The paper's experiments (Section 4) use normally distributed points, points
on low-dimensional manifolds embedded in high ambient dimension (its 1000-D
embedding of 4-D data), and Gaussian kernels with constant or per-point
bandwidth.  The recipes below keep those shapes:

* ``mixture``: a mixture of Gaussians (unit covariance, means uniform in a box).
* ``manifold``: ``x = A z + noise * e`` with ``z ~ N(0, I_k)``, ``A`` a seeded
  ``d x k`` Gaussian matrix with orthonormalised columns, ``e ~ N(0, I_d)``.

All draws use ``numpy.random.default_rng(seed)``; outputs are FP32 points and
FP32 weights.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def mixture(N: int, d: int, n_comp: int, box: float, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    means = rng.uniform(-box, box, size=(n_comp, d))
    comp = rng.integers(0, n_comp, size=N)
    X = means[comp] + rng.standard_normal((N, d))
    return X.astype(np.float32)


def manifold(N: int, d: int, k: int, noise: float, seed: int, chunk: int = 1 << 20) -> np.ndarray:
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((d, k))
    A, _ = np.linalg.qr(A)
    X = np.empty((N, d), np.float32)
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        z = rng.standard_normal((e - s, k))
        X[s:e] = (z @ A.T + noise * rng.standard_normal((e - s, d))).astype(np.float32)
    return X


def curve(N: int, d: int, seed: int) -> np.ndarray:
    """Points on the curve of Section 3's pruning experiment (intrinsic
    dimension one): x_k = f_k(k pi t), t ~ U[0, 1], k = 1..d, f_k = cos for
    odd k and sin for even k."""
    t = np.random.default_rng(seed).uniform(0.0, 1.0, N)
    k = np.arange(1, d + 1)
    arg = np.pi * t[:, None] * k[None, :]
    return np.where(k % 2 == 1, np.cos(arg), np.sin(arg)).astype(np.float32)


def gaussian(N: int, d: int, seed: int) -> np.ndarray:
    """Standard normal points (intrinsic dimension = d)."""
    return np.random.default_rng(seed).standard_normal((N, d)).astype(np.float32)


def hypersphere(N: int, d: int, seed: int) -> np.ndarray:
    """Points uniform on a hypersphere of intrinsic dimension four: the unit
    sphere of R^5 (normalized Gaussian draws) mapped into R^d by a seeded
    matrix with orthonormal columns; with d = 4 the unit sphere of R^4."""
    rng = np.random.default_rng(seed)
    k = min(5, d)
    z = rng.standard_normal((N, k))
    z /= np.linalg.norm(z, axis=1, keepdims=True)
    if k == d:
        return z.astype(np.float32)
    A, _ = np.linalg.qr(rng.standard_normal((d, k)))
    return (z @ A.T).astype(np.float32)


def manifold_queries(T: int, d: int, k: int, noise: float, seed: int, qseed: int) -> np.ndarray:
    """Fresh points from the same embedding as ``manifold(..., seed)``: the
    same matrix A (the first draw of that generator), new z and noise."""
    A = np.random.default_rng(seed).standard_normal((d, k))
    A, _ = np.linalg.qr(A)
    rng = np.random.default_rng(qseed)
    z = rng.standard_normal((T, k))
    return (z @ A.T + noise * rng.standard_normal((T, d))).astype(np.float32)


def request_stream(n: int, rate: float, seed: int, r_max: int = 64, t_min: int = 100,
                   t_max: int = 100_000) -> list[tuple[float, str, int]]:
    """Serving requests: Poisson arrivals at ``rate`` per second; each is,
    with probability 1/2, a weight request of r ~ U{1..r_max} vectors or an
    out-of-sample batch of T targets, log-uniform in [t_min, t_max].
    Returns (arrival time in s, kind, size)."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, size=n))
    out = []
    for i in range(n):
        if rng.random() < 0.5:
            out.append((float(t[i]), "weights", int(rng.integers(1, r_max + 1))))
        else:
            T = int(round(10 ** rng.uniform(np.log10(t_min), np.log10(t_max))))
            out.append((float(t[i]), "targets", T))
    return out


def weights(N: int, r: int, law: str, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed + 1000)
    if law == "normal":
        W = rng.standard_normal((N, r))
    elif law == "uniform":
        W = rng.uniform(-1.0, 1.0, size=(N, r))
    else:
        raise ValueError(law)
    return W.astype(np.float32)


@dataclass
class Workload:
    """One named workload: points, weights and the ASKIT parameters."""
    name: str
    N: int
    d: int
    points: str                 # "mixture" or "manifold"
    k_intr: int = 0             # manifold dimension
    noise: float = 0.0
    n_comp: int = 4
    box: float = 5.0
    w_law: str = "normal"
    r: int = 1
    h: float = 1.0
    leaf_size: int = 128
    kappa: int = 16
    knn_mode: int = 0           # 0 exact, 1 random-projection trees
    rp_iters: int = 4
    s_max: int = 64
    s_min: int = 1
    id_tol: float = 1e-6
    bw_mode: int = 0            # 0 constant h, 2 distance to bw_k-th neighbor
    bw_k: int = 16
    seed: int = 1
    extra: dict = field(default_factory=dict)

    def make_points(self) -> np.ndarray:
        if self.points == "mixture":
            return mixture(self.N, self.d, self.n_comp, self.box, self.seed)
        return manifold(self.N, self.d, self.k_intr, self.noise, self.seed)

    def make_weights(self, r: int | None = None, seed_offset: int = 0) -> np.ndarray:
        return weights(self.N, r or self.r, self.w_law, self.seed + seed_offset)

    def scaled(self, N: int, **kw) -> "Workload":
        d = dict(self.__dict__)
        d.update(kw)
        d["N"] = N
        d["name"] = kw.get("name", f"{self.name}@N={N}")
        return Workload(**d)


# The five workloads: a small FP64-oracle case, the 1M x 64 manifold case,
# the 8M x 64 multi-RHS case, the 1M x 1000 variable-bandwidth case and the
# 2M x 64 serving case.
SMALL_MIXTURE = Workload("mixture N=4096 d=8", 4096, 8, "mixture", n_comp=4, box=5.0,
                         h=1.0, leaf_size=128, kappa=16, knn_mode=0, s_max=64, id_tol=1e-6, seed=1)
MANIFOLD_1M_64 = Workload("manifold6 N=1048576 d=64", 1 << 20, 64, "manifold", k_intr=6,
                          noise=0.01, h=0.35, leaf_size=512, kappa=32, knn_mode=1, rp_iters=6,
                          s_max=256, id_tol=1e-4, seed=2)
MANIFOLD_8M_64_R16 = Workload("manifold10 N=8388608 d=64 r=16", 1 << 23, 64, "manifold", k_intr=10,
                              noise=0.01, w_law="uniform", r=16, h=0.5, leaf_size=1024, kappa=32,
                              knn_mode=1, rp_iters=6, s_max=512, id_tol=1e-4, seed=3)
MANIFOLD_1M_1000_VARH = Workload("manifold12 N=1048576 d=1000 var-h", 1 << 20, 1000, "manifold",
                                 k_intr=12, noise=0.001, h=1.0, leaf_size=256, kappa=16, knn_mode=1,
                                 rp_iters=4, s_max=1024, s_min=32, id_tol=1e-3, bw_mode=2, bw_k=16,
                                 seed=4)
SERVING_2M_64 = Workload("manifold8 N=2097152 d=64 serving", 1 << 21, 64, "manifold", k_intr=8,
                         noise=0.01, h=0.4, leaf_size=512, kappa=32, knn_mode=1, rp_iters=6,
                         s_max=256, id_tol=1e-4, seed=5)

ALL = [SMALL_MIXTURE, MANIFOLD_1M_64, MANIFOLD_8M_64_R16, MANIFOLD_1M_1000_VARH, SERVING_2M_64]
