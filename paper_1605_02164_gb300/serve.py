"""Request loop for the filter: continuous batching under a device-memory
budget.

Requests (one image each, with its own d, sigma_s, C, N, K, seed) arrive at any
time.  The server
  * keeps plans (sampled, whitened frequency lists) resident on the device in
    an LRU cache keyed by (d, C, sigma_s, N, K, seed, whitening); a plan evicted
    from it is destroyed only once the device is idle (destroying a plan waits
    for the device), or when many have piled up;
  * admits queued requests in arrival order while the device memory they need
    (their output buffer; inputs are the caller's) fits in the budget, and
    rejects a request larger than the whole budget (BF_ERR_BUDGET) or one whose
    window the windowed kernels cannot hold (r > BF_MAX_RADIUS: BF_ERR_UNSUPPORTED
    unless the request asks for the recursive variant);
  * launches whatever has been admitted as one bf_filter_batch call per kernel
    variant on the next free stream as soon as one is free (RGB on the tensor
    cores, other d on the FP32 kernel, or the variant a request names), so
    requests that arrive while others are on the GPU join the next batch and
    their work overlaps the batches already running (continuous batching);
  * completes requests as their batch's event fires, frees their budget and
    records per-request latency (arrival to completion);
  * lets a caller withdraw a request that is still queued (cancel).
Every filtering step runs in libbf's kernels; this module only schedules.
"""
from __future__ import annotations

import collections
import math
import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import bf

__all__ = ["Request", "Server", "summarize", "CANCELLED"]

CANCELLED = -100  # status of a request withdrawn by Server.cancel before admission


@dataclass
class Request:
    """One image to filter.  `x` is a CUDA float32 tensor (d, H, W) with unit
    column stride and a row stride that is a multiple of 4 (see
    bf.pitched_empty); the result goes to `out` (allocated on admission)."""
    x: object
    C: np.ndarray
    sigma_s: float
    K: int
    N: int = 10
    seed: int = 0
    whiten: int = bf.BF_WHITEN_CHOLESKY
    variant: int | None = None  # None: the server's choice; else a BF_* variant for this request
    t_arrival: float = 0.0
    rid: int = 0
    out: object = None
    t_admit: float = math.nan
    t_done: float = math.nan
    status: int = 1  # 1 pending, 0 done, < 0 BF_ERR_* or CANCELLED
    _bytes: int = 0
    _ready: object = None  # CUDA event on the submitting stream: x is complete once it fires
    done_evt: threading.Event = field(default_factory=threading.Event)

    @property
    def latency(self) -> float:
        return self.t_done - self.t_arrival


class Server:
    def __init__(self, budget_bytes: int = 40 << 30, streams: int = 2, max_batch: int = 64,
                 variant: int = bf.BF_FP16TC, plan_cache: int = 1024, device: int = 0, tune_cache=None):
        """tune_cache: a tune.TuneCache or the path of its JSON file; its tile
        heights go into the library's table before the loop starts, so every
        batch the loop launches takes the measured heights."""
        import torch
        self.torch = torch
        self.tuned_entries = 0
        if tune_cache is not None:
            from .tune import TuneCache
            cache = tune_cache if isinstance(tune_cache, TuneCache) else TuneCache(str(tune_cache))
            self.tuned_entries = cache.apply()
        self.dev = torch.device("cuda", device)
        self.budget = int(budget_bytes)
        self.used = 0
        self.variant = variant
        self.max_batch = max_batch
        self.streams = [torch.cuda.Stream(device=self.dev) for _ in range(streams)]
        self.busy = [None] * streams            # (event, requests) of the batch in flight per stream
        self.queue: collections.deque[Request] = collections.deque()
        self.plans: collections.OrderedDict = collections.OrderedDict()
        self.plan_cache = plan_cache
        self.retired: list[bf.Plan] = []        # evicted plans waiting for an idle device
        self.lock = threading.Lock()
        self.cv = threading.Condition(self.lock)
        self.closed = False
        self.completed: list[Request] = []
        self.rejected: list[Request] = []
        self.cancelled: list[Request] = []
        self.batches = 0
        self._thread = None

    # -- plans -------------------------------------------------------------------
    def plan(self, d: int, C, sigma_s: float, N: int, K: int, seed: int, whiten: int = 0) -> bf.Plan:
        key = (d, np.ascontiguousarray(C, np.float64).tobytes(), float(sigma_s), N, K, seed, whiten)
        p = self.plans.get(key)
        if p is None:
            p = bf.bf_plan(d, C, sigma_s, N, K, seed, whiten)
            self.plans[key] = p
            while len(self.plans) > self.plan_cache:
                self.retired.append(self.plans.popitem(last=False)[1])
            if len(self.retired) > self.plan_cache:
                self._release_retired()
        else:
            self.plans.move_to_end(key)
        return p

    def _release_retired(self):
        for p in self.retired:
            p.close()
        self.retired.clear()

    # -- client side -------------------------------------------------------------------
    def submit(self, req: Request) -> Request:
        """Queue a request.  Its input may still be in production on the caller's
        current stream: the batch that filters it waits for the work queued there
        up to this call, and the input's memory stays reserved until that batch
        has read it, even if the caller drops its reference."""
        if not req.t_arrival:
            req.t_arrival = time.perf_counter()
        torch = self.torch
        req._ready = torch.cuda.Event()
        req._ready.record(torch.cuda.current_stream(req.x.device))
        d, H, W = req.x.shape
        req._bytes = d * H * req.x.stride(1) * 4
        r = int(math.floor(3.0 * req.sigma_s + 1e-9))
        with self.cv:
            reason = None
            if req._bytes > self.budget:
                reason = bf.BF_ERR_BUDGET
            elif r > bf.BF_MAX_RADIUS and req.variant != bf.BF_FP32_RECURSIVE:
                reason = bf.BF_ERR_UNSUPPORTED  # the windowed kernels hold r <= BF_MAX_RADIUS
            if reason is not None:
                req.status = reason
                req.t_done = time.perf_counter()
                self.rejected.append(req)
                req.done_evt.set()
                return req
            self.queue.append(req)
            self.cv.notify()
        return req

    def cancel(self, req: Request) -> bool:
        """Withdraw a request that is still queued (not yet admitted): it is
        completed with status CANCELLED and no output.  Returns False when the
        request was already admitted (its batch runs to the end) or finished."""
        with self.cv:
            for i, q in enumerate(self.queue):  # by identity (requests hold tensors)
                if q is req:
                    del self.queue[i]
                    break
            else:
                return False
            req.status = CANCELLED
            req.t_done = time.perf_counter()
            self.cancelled.append(req)
            req.done_evt.set()
            return True

    def start(self):
        self._thread = threading.Thread(target=self._loop, name="bf-serve", daemon=True)
        self._thread.start()
        return self

    def close(self, wait: bool = True):
        with self.cv:
            self.closed = True
            self.cv.notify()
        if wait and self._thread:
            self._thread.join()

    # -- scheduler -----------------------------------------------------------------
    def _finish(self, i: int):
        evt, reqs = self.busy[i]
        evt.synchronize()
        now = time.perf_counter()
        with self.cv:
            for r in reqs:
                r.t_done = now
                if r.status == 1:
                    r.status = 0
                self.used -= r._bytes
                self.completed.append(r)
                r.done_evt.set()
            self.busy[i] = None

    def _admit(self) -> list[Request]:
        """Admit queued requests in arrival order while the budget allows."""
        batch = []
        with self.cv:
            while self.queue and len(batch) < self.max_batch and self.used + self.queue[0]._bytes <= self.budget:
                r = self.queue.popleft()
                self.used += r._bytes
                batch.append(r)
        return batch

    def _variant_of(self, r: Request, d: int) -> int:
        if r.variant is not None:
            return r.variant
        if self.variant in (bf.BF_FP16TC, bf.BF_BF16TC) and d not in (3, 6):
            return bf.BF_FP32  # the tensor-core kernels hold three or six channels
        return self.variant

    def _launch(self, i: int, batch: list[Request]):
        torch = self.torch
        s = self.streams[i]
        now = time.perf_counter()
        groups: dict[int, list] = {}
        with torch.cuda.stream(s):
            for r in batch:
                r.t_admit = now
                if r._ready is not None:
                    s.wait_event(r._ready)  # the input's producer work on the submitting stream
                r.x.record_stream(s)        # keep x's memory until this stream has read it
                d, H, W = r.x.shape
                r.out = torch.empty_strided(r.x.shape, r.x.stride(), dtype=torch.float32, device=self.dev)
                p = self.plan(d, r.C, r.sigma_s, r.N, r.K, r.seed, r.whiten)
                item = (p, r.x.data_ptr(), r.out.data_ptr(), H, W, r.x.stride(1))
                groups.setdefault(self._variant_of(r, d), []).append((item, r))
            for v, members in groups.items():
                try:
                    bf.bf_filter_batch([it for it, _ in members], v, s.cuda_stream)
                except bf.BFError as e:
                    for _, r in members:
                        r.status = e.code
            evt = torch.cuda.Event()
            evt.record(s)
        self.busy[i] = (evt, batch)
        self.batches += 1

    def _loop(self):
        torch = self.torch
        torch.cuda.set_device(self.dev)
        while True:
            progressed = False
            for i, b in enumerate(self.busy):
                if b is not None and b[0].query():
                    self._finish(i)
                    progressed = True
            free = [i for i, b in enumerate(self.busy) if b is None]
            if free:
                batch = self._admit()
                if batch:
                    self._launch(free[0], batch)
                    progressed = True
            if self.retired and all(b is None for b in self.busy):
                self._release_retired()  # nothing in flight: the waits cost nothing
            with self.cv:
                idle = not self.queue and all(b is None for b in self.busy)
                if self.closed and idle:
                    return
                if not progressed:
                    if not self.queue and all(b is None for b in self.busy):
                        self.cv.wait(timeout=0.01)
            if not progressed:
                time.sleep(50e-6)


def summarize(reqs: list[Request], t0: float, t1: float) -> dict:
    """Images/s, Mpixel/s and latency percentiles of completed requests."""
    done = [r for r in reqs if r.status == 0]
    lat = np.array([r.latency for r in done]) if done else np.array([math.nan])
    px = sum(r.x.shape[1] * r.x.shape[2] for r in done)
    span = max(t1 - t0, 1e-9)
    return {"completed": len(done), "rejected": sum(1 for r in reqs if r.status == bf.BF_ERR_BUDGET),
            "cancelled": sum(1 for r in reqs if r.status == CANCELLED),
            "failed": sum(1 for r in reqs if r.status < 0 and r.status not in (bf.BF_ERR_BUDGET, CANCELLED)),
            "images_per_s": len(done) / span, "mpixel_per_s": px / span / 1e6,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "span_s": span}
