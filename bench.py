#!/usr/bin/env python
"""ASKIT evaluation throughput on one GB300 (or N replicas under torchrun).

Workload: the 64-D manifold case -- N = 1,048,576 points x = A z + 0.01 e,
z ~ N(0, I_6), A a seeded 64 x 6 Gaussian matrix with orthonormal columns,
w ~ N(0, 1), Gaussian h = 0.35 (exp(-r^2 / 2h^2)), leaf size m = 512,
kappa = 32 neighbors by random-projection trees, s <= 256, ID tolerance 1e-4.

One step = one pass of the evaluation hot path over a new weight vector:
weights into tree order and the upward pass of skeleton weights, then
Evaluate at all N points, replayed as one captured CUDA graph
(askit_graph_launch; the same kernels as askit_set_weights + askit_evaluate).  The tree,
kNN, skeletons and work lists are built once (setup, reported separately).
Metric: evaluated targets per second (whole job = all ranks).

Serving (the "serving" key, 1 GPU): a 2,097,152-point 64-D tree (8-dim
manifold, h = 0.4, m = 512, s <= 256) stays resident while a seeded stream of
requests arrives as a Poisson process at 200 requests/s; each request is 1-64
new weight vectors or an out-of-sample batch of 100-100,000 points from the
same distribution.  The loop batches them continuously over two slots and
admits batches by device footprint; p50/p99 latency and targets/s are
reported for the split-precision path and for plain FP32 on the same stream.

Accuracy beside the throughput: the split path's relative error against
plain FP32 on every target (the metric's condition, <= 1e-4), ASKIT's error
eps2 and the near field's error eps_kappa against the direct sum on 1000
sampled targets, and the hit rate hr of the random-projection neighbor lists
(Section 4 reports all three).

The "prune_table" key reproduces Section 3's Table 1 (nodes visited under
distance pruning and under neighbor pruning, curve / Gaussian / hypersphere
in 2-256 dimensions, N = 65,536, m = 64, kappa = 128).

The "configs" key measures the other two benchmark workloads at full size on
the same GPU: N = 8,388,608 points in d = 64 (10-dim manifold, h = 0.5,
m = 1024, s <= 512) with r = 16 weight vectors, and N = 1,048,576 points in
d = 1000 (12-dim manifold, h_j = distance to the 16th neighbor, m = 256,
s in [32, 1024]).

--impl reference times the CPU oracle (plain FP64 C) on the host cores on a
bounded sample of the same workload and prints the same JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ASKIT eval targets/s at rel.err <=1e-4 vs plain FP32 on 1 GB300"
UNIT = "targets/s"
SM_COUNT = 152
# ex2 per SM per clock: one warp instruction per clock on the XU pipe of this
# part (ncu's XU peak; an FP16x3 Evaluate capture issues 0.436 ex2 warp
# instructions per active SM cycle and ncu reports 43.2 % of the XU peak)
MUFU_PER_SM_CLK = 32
FP32_LANES_PER_SM = 128
TF32_OVER_BF16 = 1.1 / 2.25   # nominal dense tensor-rate ratio


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16x3", choices=["simt_fp32", "tf32x3", "bf16x3", "fp16x3"])
    ap.add_argument("--workload", default="manifold1m_d64", choices=list(WORKLOADS),
                    help="which workload to time (the default is the bench line's)")
    ap.add_argument("--n", type=int, default=0, help="override N (smaller runs; not a bench line)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-n", type=int, default=0,
                    help="points of the oracle's instance (0: the workload's own N)")
    ap.add_argument("--cpu-targets", type=int, default=10000)
    ap.add_argument("--cpu-targets-1core", type=int, default=1500)
    ap.add_argument("--configs", default="auto", choices=["auto", "all", "none"],
                    help="also measure the 8M x 64 (r = 16) and 1M x 1000 (variable h) workloads at full size "
                         "(auto: with the default workload and N)")
    ap.add_argument("--serve-requests", type=int, default=200,
                    help="requests per serving run of the split path (0: no serving run)")
    ap.add_argument("--serve-requests-fp32", type=int, default=48,
                    help="requests of the saturated plain-FP32 comparator run")
    ap.add_argument("--serve-load", type=float, default=0.6,
                    help="offered load of the sustained serving run, as a fraction of the measured capacity")
    ap.add_argument("--lists", default="target", choices=["target", "leaf"],
                    help="interaction lists: per target (eq. 2.5, the bench line's) or leaf-grouped")
    return ap.parse_args()


WORKLOADS = {"manifold1m_d64": "MANIFOLD_1M_64", "manifold8m_d64_r16": "MANIFOLD_8M_64_R16",
             "manifold1m_d1000": "MANIFOLD_1M_1000_VARH"}


def workload(args):
    from paper_1410_0260_gb300 import workloads as wl
    w = getattr(wl, WORKLOADS[args.workload])
    return w.scaled(args.n) if args.n else w


def askit_config(w, precision, lists="target"):
    from paper_1410_0260_gb300 import askit
    return askit.Config(leaf_size=w.leaf_size, kappa=w.kappa, knn_mode=w.knn_mode, rp_iters=w.rp_iters,
                        s_max=w.s_max, s_min=w.s_min, id_tol=w.id_tol, h=w.h, bw_mode=w.bw_mode,
                        bw_k=w.bw_k, seed=w.seed, precision=precision, prune=2 if lists == "leaf" else 1)


def max_over_ranks(values, device):
    """Each value's maximum over the ranks (replicas do the same work, so
    the job takes as long as its slowest rank); unchanged on one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(world, n_per_rank, ms_per_step):
    """Targets per second of the whole job: every rank evaluates its own n
    targets per step (replicas, weak scaling)."""
    return world * n_per_rank / (ms_per_step / 1e3)


def roofline(P, d, r, precision, sec, peaks, smax_mhz, arg_on_tensor=False, weights_on_tensor=False,
             sustained=False):
    """Roofline of the Evaluate kernel for P algorithmic pairs in `sec`
    seconds: the binding unit among the tensor cores (three split products
    of length d per pair, and of length r when the weight sums run there
    too), MUFU (one ex2 per pair) and the FP32 FMA pipe (r FMAs per pair in
    the epilogue unless the tensor cores take the weight sums, plus 2 for the
    exponent's argument unless the tensor cores form it); plain FP32 is bound
    by its 2d lane operations per pair.  The tensor peak is the measured
    bf16 GEMM rate: the burst figure, or the sustained one (seconds of
    back-to-back GEMMs under the power cap) when the kernel is timed inside
    a long step (`sustained`, see long_step)."""
    mufu_peak = SM_COUNT * MUFU_PER_SM_CLK * smax_mhz * 1e6
    lane_peak = SM_COUNT * FP32_LANES_PER_SM * smax_mhz * 1e6
    if precision == "simt_fp32":
        # two FP32 lane operations per pair and coordinate (subtract, fused multiply-add)
        roof = {"bound": "alu", "achieved": P * 2 * d / sec / 1e12, "peak": lane_peak / 1e12,
                "unit": "Tops/s", "peak_source": "152 SMs x 128 FP32 lanes x max SM clock"}
    else:
        bf16 = ((peaks or {}).get("bf16_tflops_sustained") if sustained else None) or \
            (peaks or {}).get("bf16_tflops") or (1700.0 if sustained else 1900.0)
        tpeak = bf16 * (TF32_OVER_BF16 if precision == "tf32x3" else 1.0)   # fp16 and bf16 share the rate
        k_tensor = d + (r if weights_on_tensor else 0)     # contraction length per pair
        t_tensor = P * 3 * 2 * k_tensor / (tpeak * 1e12)
        t_mufu = P / mufu_peak
        # FP32 lane FMAs per pair in the epilogue: the exponent's argument (2)
        # and one per weight vector
        fma_per_pair = (0 if weights_on_tensor else r) + (0 if arg_on_tensor else 2)
        t_fma = P * fma_per_pair / lane_peak
        if t_fma > max(t_tensor, t_mufu):
            roof = {"bound": "alu", "achieved": P * fma_per_pair / sec / 1e12, "peak": lane_peak / 1e12,
                    "unit": "Tfma/s", "peak_source": "FP32 FMA: 152 SMs x 128 lanes x max SM clock; "
                    "%d FMAs per pair (r = %d weight sums%s)" %
                    (fma_per_pair, r, "" if arg_on_tensor else " + 2 for the exponent's argument")}
        elif t_tensor >= t_mufu:
            kind = "sustained" if sustained else "burst"
            roof = {"bound": "tensor", "achieved": P * 3 * 2 * k_tensor / sec / 1e12, "peak": tpeak, "unit": "TFLOP/s",
                    "peak_source": ("measured bf16 %s x 1.1/2.25 (TF32)" % kind if precision == "tf32x3"
                                    else "measured bf16 %s" % kind) + (" of measured" if peaks else " of fallback")}
        else:
            roof = {"bound": "alu", "achieved": P / sec / 1e12, "peak": mufu_peak / 1e12, "unit": "Tex2/s",
                    "peak_source": "MUFU ex2: 152 SMs x 32/clk x max SM clock"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    return roof


def long_step(ms_evaluate):
    """A step whose Evaluate call takes 100 ms or more keeps the GPU busy back
    to back for seconds over the warm-up and timed steps, as the sustained
    GEMM loop of the measured peaks does: its kernel is rated against the
    sustained tensor peak."""
    return ms_evaluate >= 100.0


def measured_traffic(kernel, workload_name):
    """DRAM bytes per launch of the dominant kernel from a committed ncu
    capture (profiles/traffic.json), while the kernel source is the one that
    was measured; otherwise None."""
    import hashlib
    try:
        rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json"))).get(kernel)
        if not rec or rec.get("workload") != workload_name:
            return None
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
            return None
        return rec["bytes_per_launch"]
    except (OSError, ValueError, KeyError):
        return None


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


class OracleSample:
    """The oracle as it stands, on the host cores: ASKIT setup on the
    workload itself (or, with --cpu-n, on an instance of the same recipe with
    that many points), then Evaluate (Algorithm 4) timed on a fixed sample of
    its targets."""

    def __init__(self, args, w):
        import oracle
        self.oracle = oracle
        n_pts = args.cpu_n or w.N
        ws = w if n_pts == w.N else w.scaled(n_pts)
        X, W = ws.make_points(), ws.make_weights()
        cfg = oracle.Config(leaf_size=ws.leaf_size, kappa=ws.kappa, knn_mode=ws.knn_mode,
                            rp_iters=ws.rp_iters, s_max=ws.s_max, s_min=ws.s_min, id_tol=ws.id_tol, h=ws.h,
                            bw_mode=ws.bw_mode, bw_k=ws.bw_k, seed=ws.seed)
        t0 = time.perf_counter()
        self.tree = oracle.Tree(X, cfg)
        self.tree.set_weights(W.astype(np.float64))
        self.setup_s = time.perf_counter() - t0
        n = min(args.cpu_targets, n_pts)
        self.tg = np.random.default_rng(7).choice(n_pts, size=n, replace=False)
        self.sample = (f"oracle Evaluate (Algorithm 4, FP64 C, OpenMP over targets) on {n} sampled targets of "
                       f"'{ws.name}' (N={n_pts}, d={ws.d}, m={ws.leaf_size}, kappa={ws.kappa}, s<={ws.s_max}); "
                       f"oracle setup {self.setup_s:.1f}s not timed")

    def step(self, tg=None) -> float:
        t0 = time.perf_counter()
        self.tree.evaluate(self.tg if tg is None else tg)
        return time.perf_counter() - t0

    def summary(self, seconds) -> dict:
        dt = statistics.median(seconds)
        return {"value": len(self.tg) / dt, "unit": UNIT, "cores": self.oracle.num_threads(), "kind": "oracle",
                "sample": self.sample, "seconds": dt}

    def one_core(self, n, steps=2) -> dict:
        """The same Evaluate on one host core, on the first n sampled targets."""
        cores = self.oracle.num_threads()
        tg = self.tg[:n]
        self.oracle.set_threads(1)
        try:
            dt = statistics.median([self.step(tg) for _ in range(steps)])
        finally:
            self.oracle.set_threads(cores)
        return {"value": len(tg) / dt, "unit": UNIT, "cores": 1, "targets": len(tg)}


def cpu_baseline(args, w, steps=3):
    o = OracleSample(args, w)
    out = o.summary([o.step() for _ in range(steps)])
    out["one_core"] = o.one_core(min(args.cpu_targets_1core, len(o.tg)))
    return out


def run_reference(args):
    if int(os.environ.get("RANK", "0")) != 0:
        return
    w = workload(args)
    o = OracleSample(args, w)
    for _ in range(args.warmup):
        o.step()
    base = o.summary([o.step() for _ in range(args.steps)])
    value = base["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": base["seconds"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": w.name, "N": w.N, "d": w.d, "m": w.leaf_size,
                                            "kappa": w.kappa, "s_max": w.s_max, "h": w.h},
            "cpu_baseline": {k: base[k] for k in ("value", "unit", "cores", "kind", "sample")},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


FP64_INSTR_PER_S = 0.625e12   # GB300: 1.25 TFLOP/s FP64 counted with FMAs, one instruction per clock per lane


def id_fp64_cost(tree, w, secs):
    try:
        return _id_fp64_cost(tree, w, secs)
    except Exception as e:          # a diagnostic: never lose the bench line to it
        return {"error": repr(e)}


def _id_fp64_cost(tree, w, secs):
    """FP64 operations of the skeletonization's ID (Section 2.1, as the
    kernels run it: every product and sum a separate rounded instruction, no
    FMA, so the pivots match the oracle's) from the skeleton structure, and
    their rate against GB300's FP64 instruction rate over `secs` seconds (the
    setup's skeleton stage, which also builds the node lists' samples)."""
    from paper_1410_0260_gb300 import askit
    s = tree.structure(askit.STRUCT_SKEL_S).astype(np.int64)
    c = tree.structure(askit.STRUCT_NCOL).astype(np.int64)
    N, L = w.N, tree.info()["L"]
    ops = 0.0
    for a in range(2, len(s)):
        depth = a.bit_length() - 1
        size = -(-N // (1 << depth))                   # the larger node size of the level
        ell = min(w.s_max + 20, N - size, ) if N > size else 0
        if ell <= 0 or c[a] <= 0:
            continue
        k = np.arange(min(s[a] + 1, ell, c[a]), dtype=np.float64)
        # each pivot step: trailing norms (mul + add), and for the other
        # columns the reflector's dot product and update (2 mul/add pairs)
        ops += float(np.sum(2 * (ell - k) * (c[a] - k) + 4 * (ell - k) * np.maximum(c[a] - k - 1, 0)))
        ops += float(s[a] * s[a] * (c[a] - s[a]))      # back substitution for P
        ops += float(ell * c[a] * (3 * w.d + 30))      # the kernel block: distances and the exponential
    return {"id_fp64_ops": ops, "id_fp64_instr_per_s": ops / secs if secs > 0 else None,
            "id_fp64_frac": ops / secs / FP64_INSTR_PER_S if secs > 0 else None,
            "fp64_peak_source": "1.25 TFLOP/s nominal FP64 = 0.625e12 instructions/s; the ID's canonical "
                                "arithmetic issues no FMA"}


def hit_rate(ids, ids_exact):
    """hr of Section 4: the mean fraction of the exact neighbors found."""
    hits = [len(set(a.tolist()) & set(b.tolist())) for a, b in zip(ids, ids_exact)]
    return float(np.mean(hits)) / ids.shape[1]


def accuracy(tree, precision, U, w, dev, n_sample=1000):
    """rel. L2 error of this precision against plain FP32 on every target
    (the metric's condition), ASKIT's error eps2 and the near field's error
    eps_kappa against the direct sum on sampled targets (Section 4 estimates
    both by direct evaluation at sampled points), and the hit rate hr of
    random-projection neighbor lists against the exact kNN of sampled points."""
    import torch
    from paper_1410_0260_gb300 import askit
    out = {"rel_err_vs_fp32": 0.0}
    if precision != "simt_fp32":
        tree.set_precision("simt_fp32")
        Uref = torch.empty_like(U)
        tree.kernel_timing(True)
        tree.evaluate(Uref)
        k_ms, _ = tree.kernel_timing(False)
        torch.cuda.synchronize()
        tree.set_precision(precision)
        out["fp32_kernel_ms"] = k_ms
        out["rel_err_vs_fp32"] = float(torch.linalg.vector_norm((U - Uref).double()) /
                                       torch.linalg.vector_norm(Uref.double()))
        del Uref
    N = U.shape[0]
    tg = torch.from_numpy(np.random.default_rng(11).choice(N, size=min(n_sample, N), replace=False).astype(np.int64))
    tgd = tg.to(dev)
    Udir = tree.direct(tgd)
    nd = torch.linalg.vector_norm(Udir.double())
    out["eps2_vs_direct"] = float(torch.linalg.vector_norm((U[tgd] - Udir).double()) / nd)
    Unear = tree.evaluate_part("near")
    out["eps_kappa_vs_direct"] = float(torch.linalg.vector_norm((Unear[tgd] - Udir).double()) / nd)
    del Unear
    if w.knn_mode == 1:
        ids = tg.numpy().astype(np.int32)
        exact, _ = tree.knn_points(torch.from_numpy(ids).to(dev))
        out["hr"] = hit_rate(tree.structure(askit.STRUCT_KNN)[ids], exact.cpu().numpy())
    out["sampled_targets"] = len(tg)
    return out


def extra_default(args):
    """The extra sections (Table 1, the other workloads) run with the default
    workload at full size, or when asked for."""
    return args.configs == "all" or (args.configs == "auto" and not args.n and args.workload == "manifold1m_d64")


def measure_config(args, dev, key, steps=3, warmup=2):
    """One of the other benchmark workloads at full size: setup, autotuned
    launch configuration, Evaluate time (the call and the kernel's own
    launches, CUDA events), accuracy and roofline."""
    import torch
    from paper_1410_0260_gb300 import askit
    from paper_1410_0260_gb300 import workloads as wl
    w = getattr(wl, WORKLOADS[key])
    X, W = w.make_points(), w.make_weights()
    N, r = X.shape[0], W.shape[1]
    Xd = torch.from_numpy(X).to(dev)
    Wd = torch.from_numpy(W).to(dev)
    del X
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = askit.Tree(Xd, askit_config(w, args.precision))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    del Xd
    info = tree.info()
    tree.set_weights(Wd)
    tune = tree.autotune(reps=1)
    U = torch.empty((N, r), dtype=torch.float32, device=dev)
    for _ in range(warmup):
        tree.evaluate(U)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    e0.record(stream)
    for _ in range(steps):
        tree.evaluate(U)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_eval = e0.elapsed_time(e1) / steps
    tree.kernel_timing(True)
    for _ in range(steps):
        tree.evaluate(U)
    k_ms, k_launches = tree.kernel_timing(False)
    clk = clocks.stop()
    tree.sync()
    acc = accuracy(tree, args.precision, U, w, dev)
    peaks = measured_peaks()
    g16 = args.precision == "fp16x3" and w.d <= 64 and info["fp16_centering"] == 2
    roof = roofline(info["pairs_algorithmic"], w.d, r, args.precision, k_ms / steps / 1e3, peaks,
                    (peaks or {}).get("sm_max_mhz") or 2070.0, arg_on_tensor=g16, weights_on_tensor=g16 and r > 4,
                    sustained=long_step(ms_eval))
    roof["kernel"] = ("eval_tcw_kernel" if w.d > 64 else
                      "eval_g16_kernel" if info["fp16_centering"] == 2 else "eval_tc16_kernel")
    roof["ms_per_launch"] = k_ms / max(1, k_launches)
    roof["launches_per_evaluate"] = k_launches // steps
    roof["traffic"] = measured_traffic(roof["kernel"], w.name)
    out = {"workload": w.name, "N": N, "d": w.d, "r": r, "m": w.leaf_size, "kappa": w.kappa, "s_max": w.s_max,
           "h": w.h if w.bw_mode == 0 else "distance to neighbor %d" % w.bw_k, "precision": args.precision,
           "evaluate_ms": ms_eval, "targets_per_s": N / (ms_eval / 1e3), "targets_x_rhs_per_s": N * r / (ms_eval / 1e3),
           **acc, "rel_err_ok": acc["rel_err_vs_fp32"] <= 1e-4, "roofline": roof, "clocks": clk,
           "autotune": next((c for c in tune if c["chosen"]), None),
           "fp16_centering": info["fp16_centering"], "fp16_rho": info["fp16_rho"],
           "work": {"pairs_algorithmic": info["pairs_algorithmic"], "entries": info["n_entries"],
                    "items": info["n_items"], "target_batches": info["n_batches"],
                    "near_per_target": info["near_total"] / N, "far_per_target": info["far_total"] / N,
                    "setup_s": setup_s, "setup_stage_s": {k: round(v / 1e3, 3) for k, v in info["setup_ms"].items()},
                    "skeleton_id": id_fp64_cost(tree, w, info["setup_ms"].get("skeletons", 0.0) / 1e3),
                    "device_gb": info["device_bytes"] / 1e9}}
    tree.close()
    del U, Wd
    torch.cuda.empty_cache()
    return out


def prune_table(dev, N=65536, m=64, kappa=128):
    """Section 3's Table 1: the share of tree nodes the downward pass visits,
    averaged over all targets, under distance pruning (R) and under neighbor
    pruning (kappa), for points on a curve, Gaussian points and points on a
    hypersphere of intrinsic dimension four, in 2, 4, 32 and 256 dimensions
    (N = 65,536, m = 64, kappa = 128, R unscaled)."""
    import torch
    from paper_1410_0260_gb300 import askit
    from paper_1410_0260_gb300 import workloads as wl
    out = {"N": N, "m": m, "kappa": kappa, "rscale": 1.0, "unit": "% of tree nodes visited, mean over targets"}
    t0 = time.perf_counter()
    for gen in ("curve", "gaussian", "hypersphere"):
        row = {}
        for d in (2, 4, 32, 256):
            if gen == "hypersphere" and d < 4:
                continue
            X = torch.from_numpy(getattr(wl, gen)(N, d, 17)).to(dev)
            vk, vd = askit.prune_stats(X, m, kappa, 1.0)
            L = 0
            while -(-N // (1 << L)) > m:
                L += 1
            tot = (2 << L) - 1
            row[f"{d}D"] = {"R": round(100.0 * float(vd.double().mean()) / tot, 2),
                            "kappa": round(100.0 * float(vk.double().mean()) / tot, 2)}
        out[gen] = row
    out["seconds"] = time.perf_counter() - t0
    return out


SERVE_RATE = 200.0      # arrivals per second of the serving recipe


def _mean_request_targets(N, r_max=64, t_min=100, t_max=100_000):
    """Expected evaluated targets of one request of workloads.request_stream:
    half weight requests (N r, r ~ U{1..r_max}), half target batches
    (log-uniform T in [t_min, t_max])."""
    return 0.5 * N * (r_max + 1) / 2 + 0.5 * (t_max - t_min) / np.log(t_max / t_min)


def _serve_stream(w, n, rate, seed, pool, dev):
    """n requests of the serving recipe at `rate` per second: weight requests
    take column slices of a resident pool of 128 vectors, target batches rows
    of pinned host queries (copied in by the server)."""
    import torch
    from paper_1410_0260_gb300 import workloads as wl
    spec = wl.request_stream(n, rate, seed=seed)
    rng = np.random.default_rng(seed + 17)
    n_q = sum(size for _, kind, size in spec if kind == "targets")
    Y = torch.from_numpy(wl.manifold_queries(max(n_q, 1), w.d, w.k_intr, w.noise, w.seed, seed + 99)).pin_memory()
    stream, off = [], 0
    for ta, kind, size in spec:
        if kind == "weights":
            c0 = int(rng.integers(0, 128 - size + 1))
            stream.append((ta, kind, pool[:, c0:c0 + size]))
        else:
            stream.append((ta, kind, Y[off:off + size]))
            off += size
    return stream, Y


def _serve_run(tree, Wres, stream, N, warm):
    """One replay on a fresh two-slot server: latency and throughput, the
    offered load next to the achieved one, and whether the queue grew
    (offered above what was served: the latencies then measure queueing and
    grow with the run's length)."""
    from paper_1410_0260_gb300 import serve
    srv = serve.Server(tree, Wres, n_slots=2)
    serve.replay(srv, warm)
    srv.completed.clear()
    srv.n_batches = 0
    reqs = serve.replay(srv, stream)
    st = serve.latency_stats(reqs, N)
    st["peak_concurrent_batches"] = srv.peak_concurrency
    st["batches"] = srv.n_batches
    srv.close()
    span = max(ta for ta, _, _ in stream) - min(ta for ta, _, _ in stream)
    offered = sum(N * d.shape[1] if k == "weights" else d.shape[0] for _, k, d in stream)
    st["offered_requests_per_s"] = (len(stream) - 1) / span if span > 0 else float("inf")
    st["offered_targets_per_s"] = offered / span if span > 0 else float("inf")
    st["completed_requests_per_s"] = st["completed"] / st["wall_s"]
    st["overloaded"] = bool(st["offered_targets_per_s"] > 1.1 * st["targets_per_s"])
    return st


def serving(args, dev, precision):
    """The serving workload on one resident tree: the specified stream
    (Poisson arrivals at 200/s, far above one GPU's capacity: a saturated
    run that measures capacity, its latencies are queueing), the same recipe
    at a sustainable rate (60 % of the measured capacity: the latencies of a
    stable queue), and plain FP32 saturated by the specified stream (its
    capacity, the comparator)."""
    import torch
    from paper_1410_0260_gb300 import askit
    from paper_1410_0260_gb300 import workloads as wl
    w = wl.SERVING_2M_64.scaled(2 * args.n) if args.n else wl.SERVING_2M_64
    t0 = time.perf_counter()
    tree = askit.Tree(torch.from_numpy(w.make_points()).to(dev), askit_config(w, precision))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    Wres = torch.from_numpy(w.make_weights(1)).to(dev)
    tree.set_weights(Wres)
    out_tune = tree.autotune(reps=2)
    pool = torch.from_numpy(w.make_weights(128, seed_offset=7)).to(dev)
    mean_t = _mean_request_targets(w.N)
    out = {"workload": w.name, "slots": 2, "setup_s": setup_s,
           "autotune": next((c for c in out_tune if c["chosen"]), None),
           "targets_counted_as": "N r per weight request, T per target batch",
           "mean_request_targets": mean_t}
    warm_y = torch.from_numpy(wl.manifold_queries(1000, w.d, w.k_intr, w.noise, w.seed, w.seed + 5)).pin_memory()
    warm = [(0.0, "weights", pool[:, :16]), (0.0, "targets", warm_y)]
    tree.set_precision(precision)
    stream, _ = _serve_stream(w, args.serve_requests, SERVE_RATE, w.seed, pool, dev)
    out[precision] = {"arrivals_per_s": SERVE_RATE, **_serve_run(tree, Wres, stream, w.N, warm)}
    cap = out[precision]["targets_per_s"]
    rate = args.serve_load * cap / mean_t
    stream, _ = _serve_stream(w, args.serve_requests, rate, w.seed + 1, pool, dev)
    out[precision + "_sustained"] = {"arrivals_per_s": rate, "load_of_capacity": args.serve_load,
                                     **_serve_run(tree, Wres, stream, w.N, warm)}
    if precision != "simt_fp32" and args.serve_requests_fp32 > 0:
        tree.set_precision("simt_fp32")
        stream, _ = _serve_stream(w, args.serve_requests_fp32, SERVE_RATE, w.seed, pool, dev)
        out["simt_fp32"] = {"arrivals_per_s": SERVE_RATE, **_serve_run(tree, Wres, stream, w.N, warm)}
        out["split_over_fp32_targets_per_s"] = cap / out["simt_fp32"]["targets_per_s"]
    tree.close()
    return out


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist
    from paper_1410_0260_gb300 import askit

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    w = workload(args)
    X = w.make_points()
    W = w.make_weights()
    N = w.N
    Xd = torch.from_numpy(X).to(dev)
    Wd = torch.from_numpy(W).to(dev)
    r = W.shape[1]
    U = torch.empty((N, r), dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    tree = askit.Tree(Xd, askit_config(w, args.precision, args.lists))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    info = tree.info()
    stream = torch.cuda.current_stream()

    # launch configuration of the Evaluate kernel picked by the autotuner
    # (part of setup: it times candidates on this tree's own work lists)
    tree.set_weights(Wd)
    tune = tree.autotune(reps=3)
    # the step is replayed from a captured CUDA graph (askit_graph_*): the
    # upward pass and Evaluate, one graph launch per step
    graph = tree.capture(Wd, U)
    tree.set_weights(Wd)        # the tree's default weights, for the Evaluate-only timing

    def step():
        graph.launch()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    tree.sync()
    if world > 1:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # the dominant kernel alone (Evaluate), timed on the launching stream
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    for _ in range(args.steps):
        tree.evaluate(U)
    e3.record(stream)
    torch.cuda.synchronize()
    ms_eval = e2.elapsed_time(e3) / args.steps
    # the Evaluate kernel by itself: CUDA events around each of its launches
    # on the stream it runs on (one launch per target batch)
    tree.kernel_timing(True)
    for _ in range(args.steps):
        tree.evaluate(U)
    k_ms, k_launches = tree.kernel_timing(False)
    ms_kernel = k_ms / args.steps
    clk = clocks.stop()
    tree.sync()
    # accuracy: this precision against plain FP32 on the full workload (the
    # metric's condition: rel. L2 error <= 1e-4 vs plain FP32), eps2 and
    # eps_kappa against the direct sum on 1000 sampled targets, hr
    acc = accuracy(tree, args.precision, U, w, dev)
    rel_vs_fp32 = acc["rel_err_vs_fp32"]
    ms, ms_eval, ms_kernel = max_over_ranks([ms, ms_eval, ms_kernel], dev)
    ms_step = ms / args.steps
    value = job_throughput(world, N, ms_step)

    # end to end through the public host-buffer call: H2D of w, set_weights,
    # Evaluate, D2H of u, every step
    e2e = None
    if not args.no_e2e:
        Wh = torch.from_numpy(W).pin_memory()
        Uh = torch.empty((N, r), dtype=torch.float32).pin_memory()
        for _ in range(2):
            tree.evaluate_host_ptr(Wh.data_ptr(), r, Uh.data_ptr())
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            tree.evaluate_host_ptr(Wh.data_ptr(), r, Uh.data_ptr())
        dt = time.perf_counter() - t0
        (dt,) = max_over_ranks([dt], dev)
        e2e = {"value": job_throughput(world, N, dt * 1e3 / args.steps), "unit": UNIT, "h2d_bytes_per_step": int(W.nbytes),
               "d2h_bytes_per_step": int(N * r * 4)}

    # roofline of the Evaluate kernel
    peaks = measured_peaks()
    P = info["pairs_algorithmic"]
    d = w.d
    sec = ms_kernel / 1e3
    smax = (clk or {}).get("sm_max_mhz") or (peaks or {}).get("sm_max_mhz") or 2070.0
    g16 = args.precision == "fp16x3" and d <= 64 and info["fp16_centering"] == 2
    roof = roofline(P, d, r, args.precision, sec, peaks, smax, arg_on_tensor=g16, weights_on_tensor=g16 and r > 4,
                    sustained=long_step(ms_eval))
    roof["traffic"] = None
    # the plain-FP32 comparator (the serving comparison's other side) against
    # its own roofline: one Evaluate kernel launch timed in accuracy()
    fp32_cmp = None
    if acc.get("fp32_kernel_ms"):
        rf = roofline(P, d, r, "simt_fp32", acc["fp32_kernel_ms"] / 1e3, peaks, smax)
        fp32_cmp = {"kernel": "eval_simt_kernel", "ms": acc["fp32_kernel_ms"], "roofline": rf}
    roof["kernel"] = ("eval_simt_kernel" if args.precision == "simt_fp32" else
                      "eval_tcw_kernel" if d > 64 else
                      ("eval_g16_kernel" if info["fp16_centering"] == 2 else "eval_tc16_kernel")
                      if args.precision == "fp16x3" else "eval_tc_kernel")
    roof["ms_per_launch"] = k_ms / max(1, k_launches)
    roof["launches_per_evaluate"] = k_launches // args.steps
    roof["evaluate_ms"] = ms_eval
    roof["traffic"] = measured_traffic(roof["kernel"], w.name)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(args, w)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample", "one_core")}

    # permute-in, one upward kernel per level, then per target batch Evaluate
    # and the fixed-order reduction (+ the per-sub-block column data of the
    # FP16x3 kernel)
    per_batch = 2 + (1 if (args.precision == "fp16x3" and d <= 64) else 0)
    launches_per_step = 1 + info["L"] + info["n_batches"] * per_batch
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"simt_fp32": "f32", "tf32x3": "tf32x3", "bf16x3": "bf16x3", "fp16x3": "fp16x3"}[args.precision],
            "data": "synthetic",
            "config": {"workload": w.name, "N": N, "d": d, "m": w.leaf_size, "kappa": w.kappa,
                       "knn": "rp-trees x%d" % w.rp_iters, "s_max": w.s_max, "s_min": w.s_min, "id_tol": w.id_tol,
                       "h": w.h if w.bw_mode == 0 else "distance to neighbor %d" % w.bw_k,
                       "r": r, "precision": args.precision, "parallelism": f"replicas x{world}",
                       "fp16_centering": ({1: "per source sub-block", 2: "global (data mean), pre-split"}
                                          [info["fp16_centering"]] if args.precision == "fp16x3" and d <= 64 else None),
                       "fp16_rho": info["fp16_rho"],
                       "lists": {"target": "per target (eq. 2.5)", "leaf": "leaf-grouped"}[args.lists],
                       "l2": "inputs larger than L2 (coordinates %.0f MB)" % (N * info["d_pad"] * 4 / 1e6)},
            "targets_x_rhs_per_s": value * r,
            "rel_err_vs_fp32": rel_vs_fp32, "rel_err_ok": rel_vs_fp32 <= 1e-4,
            "eps2_vs_direct": acc["eps2_vs_direct"], "eps_kappa_vs_direct": acc["eps_kappa_vs_direct"],
            "hr": acc.get("hr"),
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "clocks": clk, "roofline": roof,
            "cpu_baseline": cpu, "serving": None, "fp32_comparator": fp32_cmp,
            "autotune": {"chosen": next((c for c in tune if c["chosen"]), None), "candidates": tune},
            "work": {"pairs_algorithmic": P, "pairs_computed": info["pairs_computed"],
                     "near_per_target": info["near_total"] / N, "far_per_target": info["far_total"] / N,
                     "items": info["n_items"], "blocks": info["n_blocks"], "entries": info["n_entries"], "L": info["L"],
                     "target_batches": info["n_batches"],
                     "skeleton_rows": info["skel_total"], "setup_s": setup_s,
                     "setup_stage_s": {k: round(v / 1e3, 3) for k, v in info["setup_ms"].items()},
                     "skeleton_id": id_fp64_cost(tree, w, info["setup_ms"].get("skeletons", 0.0) / 1e3),
                     "device_gb": info["device_bytes"] / 1e9}}
    graph.close()
    tree.close()
    del Xd, Wd, U
    if rank == 0 and world == 1 and args.serve_requests > 0:
        line["serving"] = serving(args, dev, args.precision)
        if fp32_cmp:
            line["serving"]["fp32_comparator_roofline_frac"] = fp32_cmp["roofline"]["frac"]
    if rank == 0 and world == 1 and extra_default(args):
        try:
            line["prune_table"] = prune_table(dev)
        except Exception as e:
            line["prune_table"] = {"error": repr(e)}
    # the other benchmark workloads, at full size (one GPU)
    if rank == 0 and world == 1 and extra_default(args) and args.configs != "none":
        line["configs"] = {}
        for key in ("manifold8m_d64_r16", "manifold1m_d1000"):
            try:
                line["configs"][key] = measure_config(args, dev, key)
            except Exception as e:          # recorded, the main line stands
                line["configs"][key] = {"error": repr(e)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
