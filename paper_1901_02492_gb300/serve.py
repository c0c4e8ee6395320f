"""Serving loop for shift-and-stack searches: continuous admission under an HBM
budget, device-resident psi/phi while queued, overlapping execution on streams.

A request is one search job (an image stack of any size, epoch count and
velocity grid).  Its life:

  arrival -> waiting  (host FIFO)
          -> resident (admitted: its device memory fits the budget; inputs are
                       uploaded and its psi/phi planes computed on the upload
                       stream; the planes stay on the device while it queues)
          -> running  (a compute slot -- a CUDA stream -- is free: search,
                       optional FP64 rescoring, results to the host)
          -> done     (its memory and slot are released; waiting requests are
                       admitted in the same pass)

A request can be cancelled at any stage, by `Scheduler.cancel(id)` from another
thread or by its `cancel_at` time: waiting, it leaves the queue; resident, its
device memory is released (`backend.release`) without running; running, its
kernels finish (nothing stops a launch in flight) and its result is dropped.
Its Completion then has status "cancelled".  A request whose admission fails
completes with status "failed" and the error, and the loop goes on with the
others; when the failure is a shortage of device memory (the backend raises
OutOfMemory, e.g. the budget's estimate missed fragmentation) while other
requests hold memory, the request instead goes back to the head of the queue
and is admitted again after the next completion.

Admission is first-come first-served on the request's device footprint
(kb_estimate_bytes: its psi/phi planes and search buffers), so the budget is never exceeded
and a large request is not starved by smaller ones behind it.  Requests that
arrive while others run are admitted as soon as memory frees up; their
kernels overlap on the device with those already running.

The scheduler core (`Scheduler`) knows nothing of CUDA: it drives a backend
with admit / dispatch / done / finish, so its logic is tested on the CPU with a
simulated backend; `CudaBackend` runs it through the library's C ABI.
"""
from __future__ import annotations

import collections
import dataclasses
import math
import threading
import time
from typing import Any, Callable, List

import numpy as np


class OutOfMemory(MemoryError):
    """Raised by a backend's admit when device memory is short right now."""


@dataclasses.dataclass
class Request:
    id: int
    arrival: float            # seconds after the start of the run
    N: int
    H: int
    W: int
    K: int                    # PSF side
    V: int                    # velocities
    topk: int
    payload: Any = None       # what the backend needs (images, PSF, times, grid)
    nbytes: int = 0           # device footprint, set by the backend's estimate
    cancel_at: float = math.inf   # seconds after the start of the run: cancelled if not finished by then


@dataclasses.dataclass
class Completion:
    id: int
    arrival: float
    admitted: float
    started: float
    finished: float
    result: Any = None
    status: str = "done"      # "done", "cancelled" (admitted / started are nan where not reached) or "failed"

    @property
    def latency(self) -> float:
        return self.finished - self.arrival


class Scheduler:
    """Continuous admission and dispatch of requests onto `slots` compute slots
    under a device-memory budget of `budget` bytes.

    Admission to device memory is first-come first-served.  Dispatch of resident
    requests to a free slot follows `policy`:
      "fifo"  in admission order;
      "sjf"   least work first (trajectory-epoch evaluations N H W V), except that
              a request resident for longer than `max_wait` seconds goes first
              (oldest first), so large requests are delayed, never starved."""

    def __init__(self, backend, budget: int, slots: int = 4, poll_s: float = 2e-4, policy: str = "fifo",
                 max_wait: float = 2.0):
        if policy not in ("fifo", "sjf"):
            raise ValueError("unknown policy %r" % policy)
        self.backend = backend
        self.budget = int(budget)
        self.slots = int(slots)
        self.poll_s = poll_s
        self.policy = policy
        self.max_wait = float(max_wait)
        self.peak_bytes = 0
        self._lock = threading.Lock()
        self._cancel = set()

    def cancel(self, request_id: int):
        """Cancel a request (any thread, any time during or before `run`)."""
        with self._lock:
            self._cancel.add(int(request_id))

    def _next(self, resident, now):
        """Index in `resident` of the request to dispatch next."""
        if self.policy == "fifo":
            return 0
        overdue = [i for i, (r, h, t_adm) in enumerate(resident) if now - t_adm > self.max_wait]
        if overdue:
            return overdue[0]
        return min(range(len(resident)), key=lambda i: (work(resident[i][0]), resident[i][0].arrival,
                                                         resident[i][0].id))

    def run(self, requests: List[Request], clock: Callable[[], float] = time.perf_counter,
            sleep: Callable[[float], None] = time.sleep) -> List[Completion]:
        be = self.backend
        for r in requests:
            r.nbytes = be.estimate(r)
            if r.nbytes > self.budget:
                raise ValueError("request %d needs %d bytes, more than the whole budget %d"
                                 % (r.id, r.nbytes, self.budget))
        pending = collections.deque(sorted(requests, key=lambda r: (r.arrival, r.id)))
        waiting: collections.deque = collections.deque()
        resident: collections.deque = collections.deque()
        running = {}                                   # slot -> (request, handle, admitted, started)
        free_slots = list(range(self.slots))[::-1]
        in_use = 0
        out: List[Completion] = []
        deadlines = any(math.isfinite(r.cancel_at) for r in requests)
        dropping = set()                               # running requests whose result is dropped
        retry_blocked = False                          # an admission ran out of memory: wait for a completion
        t0 = clock()
        while pending or waiting or resident or running:
            now = clock() - t0
            progressed = False
            with self._lock:
                ids = set(self._cancel)
            if ids or deadlines:
                def gone(r):
                    return r.id in ids or now >= r.cancel_at
                for q in (pending, waiting):
                    for r in [r for r in q if gone(r)]:
                        q.remove(r)
                        out.append(Completion(r.id, r.arrival, math.nan, math.nan, now, None, "cancelled"))
                        progressed = True
                for item in [x for x in resident if gone(x[0])]:
                    r, h, t_adm = item
                    resident.remove(item)
                    be.release(h)
                    in_use -= r.nbytes
                    retry_blocked = False
                    out.append(Completion(r.id, r.arrival, t_adm, math.nan, clock() - t0, None, "cancelled"))
                    progressed = True
                for slot, (r, h, t_adm, t_start) in running.items():
                    if gone(r):
                        dropping.add(r.id)
            while pending and pending[0].arrival <= now:
                waiting.append(pending.popleft())
                progressed = True
            for slot in list(running):
                r, h, t_adm, t_start = running[slot]
                if be.done(h):
                    res = be.finish(h)
                    t_fin = clock() - t0
                    if r.id in dropping:
                        out.append(Completion(r.id, r.arrival, t_adm, t_start, t_fin, None, "cancelled"))
                    else:
                        out.append(Completion(r.id, r.arrival, t_adm, t_start, t_fin, res))
                    in_use -= r.nbytes
                    del running[slot]
                    free_slots.append(slot)
                    retry_blocked = False
                    progressed = True
            while waiting and in_use + waiting[0].nbytes <= self.budget and not retry_blocked:
                r = waiting.popleft()
                try:
                    h = be.admit(r)
                except OutOfMemory as e:               # the backend released what it had taken
                    if resident or running:
                        waiting.appendleft(r)          # again after the next completion
                        retry_blocked = True
                        continue
                    out.append(Completion(r.id, r.arrival, math.nan, math.nan, clock() - t0, e, "failed"))
                    progressed = True
                    continue
                except Exception as e:
                    out.append(Completion(r.id, r.arrival, math.nan, math.nan, clock() - t0, e, "failed"))
                    progressed = True
                    continue
                in_use += r.nbytes
                self.peak_bytes = max(self.peak_bytes, in_use)
                resident.append((r, h, clock() - t0))
                progressed = True
            while resident and free_slots:
                i = self._next(resident, clock() - t0)
                r, h, t_adm = resident[i]
                del resident[i]
                slot = free_slots.pop()
                be.dispatch(h, slot)
                running[slot] = (r, h, t_adm, clock() - t0)
                progressed = True
            if not progressed:
                wait = self.poll_s
                if pending and not (waiting or resident or running):
                    wait = max(0.0, min(0.05, pending[0].arrival - (clock() - t0)))
                sleep(wait)
        return out


def work(r: Request) -> int:
    """Trajectory-epoch evaluations of a request's search."""
    return r.N * r.H * r.W * r.V


def fifo_latencies(arrivals: np.ndarray, service: np.ndarray) -> np.ndarray:
    """Latencies of a single server that takes requests one at a time in arrival
    order, each for its measured service time (the serial baseline)."""
    lat = np.empty(len(arrivals))
    free_at = 0.0
    for i, (a, s) in enumerate(zip(arrivals, service)):
        start = max(a, free_at)
        free_at = start + s
        lat[i] = free_at - a
    return lat


def busy_fraction(intervals) -> float:
    """Fraction of [first start, last end] covered by the union of (start, end) intervals."""
    iv = sorted(intervals)
    if not iv:
        return 0.0
    total, cur_s, cur_e = 0.0, iv[0][0], iv[0][1]
    for s, e in iv[1:]:
        if s > cur_e:
            total += cur_e - cur_s
            cur_s, cur_e = s, e
        else:
            cur_e = max(cur_e, e)
    total += cur_e - cur_s
    span = max(e for _, e in iv) - iv[0][0]
    return total / span if span > 0 else 0.0


class CudaBackend:
    """Runs requests through the library: kb_stack (psi/phi) on an upload stream,
    kb_job search (+ FP64 rescoring) and results on one stream per slot.

    A request's payload is a dict with host arrays `sci`, `var` ([>= N][H][W]
    float32, pinned torch tensors; the first N epochs are used), `psf`
    ([N][K][K]), `times` [N], `vx`, `vy` [V].  All buffers that outlive a
    request are allocated up front, so the loop itself allocates only through
    the library's stream-ordered pool: the device input staging (reused in
    upload-stream order) and, per slot, a device and a pinned host buffer for
    the results (kb_result records; returned as [H][W][topk] with keep_results).
    """

    def __init__(self, ctx, device, storage: str = "bf16", rescore: bool = True, slots: int = 4,
                 max_npix: int = 1, max_planes: int = 1, max_topk: int = 16, keep_results: bool = False,
                 time_device: bool = True):
        import torch
        from . import binding as kb
        self.kb, self.torch = kb, torch
        self.ctx = ctx
        self.dev = device
        self.storage = storage
        self.flags = kb.KB_RESCORE_FP64 if rescore else 0
        self.keep = keep_results
        self.time_device = time_device
        self.upload = torch.cuda.Stream(device)
        self.streams = [torch.cuda.Stream(device) for _ in range(slots)]
        self.max_planes = max_planes
        self.stage = torch.empty(2 * max_planes, dtype=torch.float32, device=device)
        rb = max_npix * max_topk * kb.RESULT_DTYPE.itemsize
        self.dev_out = [torch.empty(rb, dtype=torch.uint8, device=device) for _ in range(slots)]
        self.host_out = [torch.empty(rb, dtype=torch.uint8).pin_memory() for _ in range(slots)]
        self.ref = torch.cuda.Event(enable_timing=True)
        self.ref.record(self.upload)
        self.intervals_ev = []
        torch.cuda.synchronize(device)

    @property
    def fixed_bytes(self) -> int:
        """Device bytes the backend holds outside any request: input staging and result buffers."""
        return self.stage.numel() * 4 + sum(b.numel() for b in self.dev_out)

    def estimate(self, r: Request) -> int:
        s, j = self.kb.estimate_bytes(r.N, r.H, r.W, self.storage, r.K, r.V, r.topk, self.flags)
        return s + j

    def admit(self, r: Request):
        kb, torch = self.kb, self.torch
        p = r.payload
        n = r.N * r.H * r.W
        if n > self.max_planes or r.H * r.W * r.topk * kb.RESULT_DTYPE.itemsize > self.dev_out[0].numel():
            raise ValueError("request %d is larger than the backend's staging" % r.id)
        try:
            st = kb.Stack(self.ctx, r.N, r.H, r.W, self.storage)
        except kb.KBError as e:
            if e.code == kb.KB_ENOMEM:
                raise OutOfMemory(str(e)) from e
            raise
        job = None
        try:                                  # on failure, free what this admission took
            job = kb.Job(self.ctx, r.H, r.W, r.N, r.V, r.topk, self.flags)
            with torch.cuda.stream(self.upload):
                sci = self.stage[:n].view(r.N, r.H, r.W)
                var = self.stage[self.max_planes:self.max_planes + n].view(r.N, r.H, r.W)
                sci.copy_(p["sci"][:r.N], non_blocking=True)
                var.copy_(p["var"][:r.N], non_blocking=True)
                st.make_psi_phi(sci, var, None, p["psf"][:r.N], stream=self.upload)
                ready = torch.cuda.Event()
                ready.record(self.upload)
        except Exception as e:
            self.upload.synchronize()
            if job is not None:
                job.free()
            st.free()
            if isinstance(e, kb.KBError) and e.code == kb.KB_ENOMEM:
                raise OutOfMemory(str(e)) from e
            raise
        return dict(r=r, stack=st, job=job, ready=ready, done=None)

    def dispatch(self, h, slot: int):
        torch = self.torch
        r, p = h["r"], h["r"].payload
        s = self.streams[slot]
        nbytes = r.H * r.W * r.topk * self.kb.RESULT_DTYPE.itemsize
        out, host = self.dev_out[slot][:nbytes], self.host_out[slot][:nbytes]
        s.wait_event(h["ready"])
        t0 = torch.cuda.Event(enable_timing=True) if self.time_device else None
        t1 = torch.cuda.Event(enable_timing=True) if self.time_device else None
        with torch.cuda.stream(s):
            if t0 is not None:
                t0.record(s)
            h["job"].search(h["stack"], p["times"][:r.N], p["vx"], p["vy"], r.topk, -math.inf, self.flags, stream=s)
            h["job"].results(out, stream=s)
            host.copy_(out, non_blocking=True)
            if t1 is not None:
                t1.record(s)
            done = torch.cuda.Event()
            done.record(s)
        h["done"], h["slot"], h["nbytes"] = done, slot, nbytes
        if t0 is not None:
            self.intervals_ev.append((t0, t1))

    def done(self, h) -> bool:
        return h["done"].query()

    def release(self, h):
        """Free an admitted request that will not run (cancelled while resident)."""
        h["ready"].synchronize()              # its uploads and psi/phi are done with the staging
        h["job"].free()
        h["stack"].free()

    def finish(self, h):
        h["job"].wait()                       # raises on a device-side status
        res = None
        if self.keep:
            r = h["r"]
            res = (self.host_out[h["slot"]][:h["nbytes"]].numpy().copy()
                   .view(self.kb.RESULT_DTYPE).reshape(r.H, r.W, r.topk))
        h["job"].free()
        h["stack"].free()
        return res

    def device_intervals(self):
        """(start, end) of every dispatched request's device work, seconds after the backend started."""
        self.torch.cuda.synchronize(self.dev)
        return [(self.ref.elapsed_time(a) * 1e-3, self.ref.elapsed_time(b) * 1e-3) for a, b in self.intervals_ev]
