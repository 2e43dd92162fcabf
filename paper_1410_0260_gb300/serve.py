"""Serving loop over a skeletonized ASKIT tree resident on the GPU.

Requests are either new weight vectors W [N, r] (answer: u = K~ W at every
point, Algorithm 4) or a batch of out-of-sample targets Y [T, d] (answer: u at
those targets with the resident weights).  A scheduler thread batches the
waiting requests continuously -- weight requests are merged column-wise up to
`max_r` columns (larger requests are split into column chunks), target
requests are concatenated up to `max_T` rows -- and hands each batch to a free
slot.  A slot owns a CUDA stream and a weight context (askit_weights_*), so
batches on different slots overlap on the device while the tree is shared.  A
batch is admitted only when its device-memory footprint (askit_footprint)
fits the remaining budget; requests that can never fit are rejected.

Every GPU step of a batch runs in the C library; this module only moves
requests between threads.

Latency is measured per request from submission to the host copy of its
result; `t_start` marks when its batch left the queue, so queueing delay and
service time can be told apart.
"""
from __future__ import annotations

import contextlib
import threading
import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np
import torch

from . import askit


@dataclass(eq=False)          # requests compare by identity
class Request:
    kind: str                 # "weights" or "targets"
    data: torch.Tensor        # W [N, r] or Y [T, d], FP32 (host or device)
    t_arrival: float = 0.0
    t_start: float = 0.0
    t_done: float = 0.0
    result: torch.Tensor | None = None
    error: str | None = None
    done: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class _Slot:
    def __init__(self, tree: askit.Tree, device):
        self.stream = torch.cuda.Stream(device=device) if device.type == "cuda" else None
        self.ctx = tree.weights_context()
        self.busy = False


class Server:
    def __init__(self, tree: askit.Tree, resident_W: torch.Tensor, n_slots: int = 2,
                 budget_bytes: int | None = None, max_r: int = 16, max_cols: int = 64,
                 max_T: int = 131072):
        """max_r: columns per evaluation (the tensor-core path covers r <= 16);
        max_cols: columns of one merged weight batch (evaluated in chunks of
        max_r); max_T: targets of one merged out-of-sample batch."""
        self.tree = tree
        self.device = tree.device
        self.max_r, self.max_cols, self.max_T = max_r, max_cols, max_T
        self.resident = tree.weights_context()
        self.resident.set(resident_W.to(self.device))
        if self.device.type == "cuda":
            torch.cuda.synchronize(self.device)
        if budget_bytes is None:
            free, _ = torch.cuda.mem_get_info(self.device)
            budget_bytes = int(free * 0.8)
        self.budget = budget_bytes
        self.free_bytes = budget_bytes
        self.slots = [_Slot(tree, self.device) for _ in range(n_slots)]
        self.queue: deque[Request] = deque()
        self.cv = threading.Condition()
        self.stop = False
        self.completed: list[Request] = []
        self.peak_concurrency = 0
        self.n_batches = 0
        self._sched = threading.Thread(target=self._schedule, daemon=True)
        self._sched.start()

    # ------------------------------------------------------------------ API
    def submit(self, req: Request) -> Request:
        req.t_arrival = time.perf_counter()
        with self.cv:
            self.queue.append(req)
            self.cv.notify_all()
        return req

    def close(self):
        with self.cv:
            self.stop = True
            self.cv.notify_all()
        self._sched.join()
        for s in self.slots:
            if s.stream is not None:
                s.stream.synchronize()
            s.ctx.close()
        self.resident.close()

    # ------------------------------------------------------------- batching
    def batch_bytes(self, kind: str, n: int) -> int:
        """Device bytes of one batch: n columns of weights, or n targets."""
        return batch_bytes(self.tree, kind, n, self.max_r, self.resident.r)

    def _take_batch(self):
        """Oldest request first; merge following requests of the same kind
        while the merged batch stays within the size caps and the budget."""
        head = self.queue[0]
        batch = [head]
        if head.kind == "weights":
            n, cap, dim = head.data.shape[1], self.max_cols, 1
        else:
            n, cap, dim = head.data.shape[0], self.max_T, 0
        need = self.batch_bytes(head.kind, n)
        for q in list(self.queue)[1:]:
            if q.kind != head.kind or n + q.data.shape[dim] > cap:
                continue
            nq = self.batch_bytes(head.kind, n + q.data.shape[dim])
            if nq > self.budget:
                continue
            batch.append(q)
            n += q.data.shape[dim]
            need = nq
        return batch, need

    def _schedule(self):
        try:
            self._schedule_loop()
        except Exception as e:          # a scheduler failure fails every waiting request
            with self.cv:
                self.stop = True
                while self.queue:
                    r = self.queue.popleft()
                    r.error = f"scheduler failed: {e!r}"
                    r.t_done = time.perf_counter()
                    r.done.set()

    def _schedule_loop(self):
        while True:
            with self.cv:
                while not self.stop and (not self.queue or not any(not s.busy for s in self.slots)):
                    self.cv.wait()
                if self.stop and not self.queue:
                    return
                batch, need = self._take_batch()
                if need > self.budget:
                    # can never fit: reject the oldest request
                    r = self.queue.popleft()
                    r.error = f"request needs {need} device bytes, budget is {self.budget}"
                    r.t_done = time.perf_counter()
                    r.done.set()
                    continue
                while need > self.free_bytes and not self.stop:
                    self.cv.wait()        # admission: wait for memory to free up
                t = time.perf_counter()
                taken = {id(r) for r in batch}
                self.queue = deque(q for q in self.queue if id(q) not in taken)
                for r in batch:
                    r.t_start = t
                slot = next(s for s in self.slots if not s.busy)
                slot.busy = True
                self.n_batches += 1
                self.free_bytes -= need
                self.peak_concurrency = max(self.peak_concurrency, sum(s.busy for s in self.slots))
            threading.Thread(target=self._run, args=(slot, batch, need), daemon=True).start()

    def _run(self, slot: _Slot, batch: list[Request], need: int):
        try:
            with torch.cuda.stream(slot.stream) if slot.stream is not None else contextlib.nullcontext():
                if batch[0].kind == "weights":
                    W = torch.cat([r.data.to(self.device, non_blocking=True) for r in batch], dim=1)
                    outs = []
                    for c0 in range(0, W.shape[1], self.max_r):     # column chunks of max_r
                        slot.ctx.set(W[:, c0:c0 + self.max_r].contiguous(), stream=slot.stream)
                        outs.append(slot.ctx.evaluate(stream=slot.stream))
                    U = torch.cat(outs, dim=1).cpu()
                    c = 0
                    for r in batch:
                        k = r.data.shape[1]
                        r.result = U[:, c:c + k]
                        c += k
                else:
                    Y = torch.cat([r.data.to(self.device, non_blocking=True) for r in batch], dim=0)
                    U = self.resident.evaluate_targets(Y, stream=slot.stream).cpu()
                    c = 0
                    for r in batch:
                        k = r.data.shape[0]
                        r.result = U[c:c + k]
                        c += k
            if slot.stream is not None:
                slot.stream.synchronize()
        except Exception as e:          # report per request, keep serving
            for r in batch:
                r.error = str(e)
        t = time.perf_counter()
        with self.cv:
            for r in batch:
                r.t_done = t
                self.completed.append(r)
                r.done.set()
            slot.busy = False
            self.free_bytes += need
            self.cv.notify_all()


def batch_bytes(tree: askit.Tree, kind: str, n: int, max_r: int = 16, r_resident: int = 1) -> int:
    """Device footprint of a batch: the library's estimate of its working
    memory (askit_footprint) plus the request data and results held by the
    serving loop."""
    if kind == "weights":
        return tree.footprint(0, 0, min(n, max_r)) + 2 * 4 * tree.N * n
    return tree.footprint(1, n, r_resident) + 4 * n * (tree.d + r_resident)


def replay(server: Server, stream: list[tuple[float, str, torch.Tensor]], timeout: float = 600.0) -> list[Request]:
    """Submit (arrival time in s, kind, data) requests at their arrival times
    and wait for all of them (at most `timeout` seconds in all)."""
    reqs = []
    t0 = time.perf_counter()
    for ta, kind, data in stream:
        dt = t0 + ta - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        reqs.append(server.submit(Request(kind, data)))
    deadline = time.perf_counter() + timeout
    for r in reqs:
        if not r.done.wait(max(0.0, deadline - time.perf_counter())):
            raise TimeoutError("serving replay did not finish in %.0f s" % timeout)
    return reqs


def latency_stats(reqs: list[Request], N: int, r_resident: int = 1) -> dict:
    """p50/p99 latency (submission to result on the host), service time and
    throughput in evaluated targets per second: a weight request of r vectors
    counts N r targets, a target batch of T points counts T r_resident."""
    ok = [r for r in reqs if r.error is None]
    lat = np.array([r.latency for r in ok]) * 1e3
    svc = np.array([r.t_done - r.t_start for r in ok]) * 1e3
    t0 = min(r.t_arrival for r in reqs)
    t1 = max(r.t_done for r in reqs)
    targets = sum(N * r.data.shape[1] if r.kind == "weights" else r.data.shape[0] * r_resident for r in ok)
    return {"requests": len(reqs), "completed": len(ok), "rejected": len(reqs) - len(ok),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "service_p50_ms": float(np.percentile(svc, 50)), "service_p99_ms": float(np.percentile(svc, 99)),
            "targets_per_s": targets / (t1 - t0), "wall_s": t1 - t0}
