"""The serving scheduler's host logic on a simulated backend (no GPU).

The backend simulates a device whose requests each take a fixed service time
once dispatched and run side by side on the slots; the scheduler is driven by a
virtual clock.  Checked: the memory budget is never exceeded, admission is in
arrival order, at most `slots` requests run at once, requests arriving while
others run are admitted as soon as memory allows, every request completes
once, the serial-baseline and busy-fraction arithmetic, and the host-side
failure paths: cancellation of waiting, resident and running requests, failed
admissions (a malformed request, an allocation failure under a fake budget).
"""
import math

import numpy as np
import pytest

from paper_1901_02492_gb300.serve import OutOfMemory, Request, Scheduler, busy_fraction, fifo_latencies


class Clock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class SimBackend:
    def __init__(self, clock, service):
        self.clock, self.service = clock, service
        self.in_use = 0
        self.max_in_use = 0
        self.running = 0
        self.max_running = 0
        self.admitted = []
        self.events = []
        self.finished = []
        self.released = []

    def estimate(self, r):
        return r.N * r.H * r.W

    def admit(self, r):
        self.in_use += r.nbytes
        self.max_in_use = max(self.max_in_use, self.in_use)
        self.admitted.append(r.id)
        self.clock.t += 1e-4                      # host cost of an admission
        return {"r": r}

    def dispatch(self, h, slot):
        self.running += 1
        self.max_running = max(self.max_running, self.running)
        h["end"] = self.clock() + self.service(h["r"])
        h["slot"] = slot

    def done(self, h):
        return self.clock() >= h["end"]

    def finish(self, h):
        self.running -= 1
        self.in_use -= h["r"].nbytes
        self.finished.append(h["r"].id)
        return h["r"].id

    def release(self, h):
        self.in_use -= h["r"].nbytes
        self.released.append(h["r"].id)


class FaultyBackend(SimBackend):
    """Admission fails for a malformed request (payload "bad") and, like a device
    whose allocator runs out first, when the memory taken would pass `device_bytes`
    (a fake budget below the scheduler's); a failed admission takes nothing."""

    def __init__(self, clock, service, device_bytes):
        super().__init__(clock, service)
        self.device_bytes = device_bytes

    def admit(self, r):
        if r.payload == "bad":
            raise ValueError("malformed request %d" % r.id)
        if self.in_use + r.nbytes > self.device_bytes:
            raise OutOfMemory("out of device memory for request %d" % r.id)
        return super().admit(r)


def _requests(n, seed=0, rate=50.0):
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    sizes = [(8, 8), (32, 64), (64, 64)]
    out = []
    for i in range(n):
        H, W = sizes[int(rng.integers(0, 3))]
        out.append(Request(i, float(t[i]), int(rng.integers(5, 16)), H, W, 7, 256, 8))
    return out


@pytest.mark.parametrize("slots,budget", [(1, 70000), (4, 70000), (4, 200000), (8, 61440)])
def test_budget_slots_and_order(slots, budget):
    clk = Clock()
    be = SimBackend(clk, lambda r: 1e-6 * r.H * r.W * r.N / 10)
    reqs = _requests(300)
    out = Scheduler(be, budget, slots).run(reqs, clock=clk, sleep=clk.sleep)
    assert sorted(c.id for c in out) == list(range(300))
    assert be.max_in_use <= budget
    assert be.max_running <= slots
    assert be.admitted == sorted(be.admitted, key=lambda i: (reqs[i].arrival, i))   # FIFO admission
    for c in out:
        r = reqs[c.id]
        assert c.arrival <= c.admitted <= c.started <= c.finished
        assert c.finished - c.started >= 1e-6 * r.H * r.W * r.N / 10 - 1e-9
    assert be.in_use == 0 and be.running == 0


def test_requests_join_while_others_run():
    """Continuous batching: a request arriving during a long one starts before it ends."""
    clk = Clock()
    long_r = Request(0, 0.0, 10, 64, 64, 7, 256, 8)
    short = [Request(i, 0.01 * i, 5, 8, 8, 7, 256, 8) for i in range(1, 6)]
    be = SimBackend(clk, lambda r: 1.0 if r.id == 0 else 0.002)
    out = {c.id: c for c in Scheduler(be, 10 ** 6, 4).run([long_r] + short, clock=clk, sleep=clk.sleep)}
    for i in range(1, 6):
        assert out[i].started < out[0].finished
        assert out[i].latency < 0.1


def test_admission_waits_for_memory_and_does_not_starve_large_requests():
    clk = Clock()
    big = Request(1, 0.001, 10, 100, 100, 7, 256, 8)          # 100000 bytes: the whole budget
    small = [Request(0, 0.0, 5, 10, 10, 7, 256, 8)] + [Request(i, 0.001 + 1e-4 * i, 5, 10, 10, 7, 256, 8)
                                                        for i in range(2, 30)]
    be = SimBackend(clk, lambda r: 0.01)
    out = {c.id: c for c in Scheduler(be, 100000, 4).run([big] + small, clock=clk, sleep=clk.sleep)}
    assert be.max_in_use <= 100000
    # the big request waits only for request 0 to leave, and no later small request overtakes it
    assert out[1].admitted >= out[0].finished
    assert all(out[i].admitted >= out[1].finished for i in range(2, 30))


def test_request_larger_than_budget_is_rejected():
    clk = Clock()
    be = SimBackend(clk, lambda r: 0.01)
    with pytest.raises(ValueError):
        Scheduler(be, 1000, 2).run([Request(0, 0.0, 10, 64, 64, 7, 256, 8)], clock=clk, sleep=clk.sleep)


def test_fifo_latencies_and_busy_fraction():
    arr = np.array([0.0, 0.5, 0.6, 5.0])
    svc = np.array([1.0, 1.0, 1.0, 0.5])
    # starts 0, 1, 2, 5 -> ends 1, 2, 3, 5.5
    assert np.allclose(fifo_latencies(arr, svc), [1.0, 1.5, 2.4, 0.5])
    assert busy_fraction([(0, 1), (0.5, 2), (3, 4)]) == pytest.approx(3.0 / 4.0)
    assert busy_fraction([(0, 1), (1, 2)]) == pytest.approx(1.0)
    assert busy_fraction([]) == 0.0


def test_sjf_dispatch_serves_small_jobs_first_and_bounds_waiting():
    """Least work first among resident requests, with the aging bound: a request
    resident longer than max_wait is dispatched before any newer one."""
    from paper_1901_02492_gb300.serve import work
    clk = Clock()
    big = [Request(i, 0.0, 10, 64, 64, 7, 256, 8) for i in range(3)]
    small = [Request(10 + i, 0.001 * i, 5, 8, 8, 7, 256, 8) for i in range(20)]
    be = SimBackend(clk, lambda r: 1e-6 * work(r) / 256)
    out = {c.id: c for c in Scheduler(be, 10 ** 9, 1, policy="sjf", max_wait=0.25).run(big + small, clock=clk,
                                                                                        sleep=clk.sleep)}
    assert sorted(out) == sorted(r.id for r in big + small)
    # request 0 started first (alone in the queue); afterwards small ones overtake the big ones
    first_small = min(out[10 + i].started for i in range(20))
    assert first_small < out[1].started
    # no big request waits past the bound plus one running job's service time
    svc_big = 1e-6 * work(big[0]) / 256
    for r in big:
        assert out[r.id].started - out[r.id].admitted <= 0.25 + svc_big + 0.01
    # FIFO on the same input dispatches in admission order
    clk2 = Clock()
    be2 = SimBackend(clk2, lambda r: 1e-6 * work(r) / 256)
    fifo = Scheduler(be2, 10 ** 9, 1, policy="fifo").run(big + small, clock=clk2, sleep=clk2.sleep)
    starts = [c.id for c in sorted(fifo, key=lambda c: c.started)]
    assert starts == [r.id for r in sorted(big + small, key=lambda r: (r.arrival, r.id))]


def test_sjf_lowers_median_latency_on_a_mixed_stream():
    from paper_1901_02492_gb300.serve import work
    reqs = _requests(400, seed=5, rate=60.0)
    res = {}
    for policy in ("fifo", "sjf"):
        clk = Clock()
        be = SimBackend(clk, lambda r: 2e-6 * r.H * r.W * r.N / 10)
        done = Scheduler(be, 200000, 2, policy=policy).run([Request(**vars(r)) for r in reqs], clock=clk,
                                                            sleep=clk.sleep)
        assert be.max_in_use <= 200000
        res[policy] = np.median([c.latency for c in done])
    assert res["sjf"] <= res["fifo"]


def test_cancel_mid_queue_resident_and_running():
    """One slot, budget for two requests: request 0 runs, 1 is resident, 2-5 wait.
    Cancelled by time: 3 while waiting, 1 while resident, 0 while running; request
    4 by Scheduler.cancel from the clock (another caller) while waiting."""
    clk = Clock()
    reqs = [Request(i, 0.001 * i, 5, 10, 10, 7, 256, 8) for i in range(6)]      # 500 bytes each
    reqs[3].cancel_at = 0.05
    reqs[1].cancel_at = 0.2
    reqs[0].cancel_at = 0.5
    be = SimBackend(clk, lambda r: 1.0)
    sched = Scheduler(be, 1000, 1)

    def sleep(dt):
        clk.sleep(dt)
        if clk.t >= 0.1:
            sched.cancel(4)

    out = {c.id: c for c in sched.run(reqs, clock=clk, sleep=sleep)}
    assert sorted(out) == list(range(6))
    assert [out[i].status for i in range(6)] == ["cancelled", "cancelled", "done", "cancelled", "cancelled", "done"]
    # 0 ran to the end of its kernels, its result dropped; 1 was released without running
    assert out[0].result is None and 0 in be.finished and out[0].finished >= 1.0
    assert be.released == [1] and math.isnan(out[1].started) and out[1].finished < 1.0
    # 3 and 4 never reached the device
    assert 3 not in be.admitted and 4 not in be.admitted
    assert math.isnan(out[3].admitted) and 0.05 <= out[3].finished < 0.1
    assert out[2].result == 2 and out[5].result == 5
    assert be.in_use == 0 and be.running == 0 and be.max_in_use <= 1000


def test_cancel_before_arrival():
    clk = Clock()
    reqs = [Request(0, 0.0, 5, 10, 10, 7, 256, 8), Request(1, 0.5, 5, 10, 10, 7, 256, 8)]
    be = SimBackend(clk, lambda r: 0.01)
    sched = Scheduler(be, 10 ** 6, 2)
    sched.cancel(1)
    out = {c.id: c for c in sched.run(reqs, clock=clk, sleep=clk.sleep)}
    assert out[0].status == "done" and out[1].status == "cancelled" and be.admitted == [0]


def test_failed_admissions_complete_and_the_rest_run():
    """A malformed request completes as "failed" with the error; requests whose
    allocation fails (the device holds less than the scheduler's budget) go back to
    the head of the queue and run after the next completion; one that cannot fit
    even alone fails.  Nothing a failed admission took stays taken."""
    clk = Clock()
    reqs = [Request(i, 0.001 * i, 5, 10, 10, 7, 256, 8) for i in range(8)]     # 500 bytes each
    reqs[2].payload = "bad"
    be = FaultyBackend(clk, lambda r: 0.05 if r.id else 0.2, device_bytes=1000)
    out = {c.id: c for c in Scheduler(be, 1500, 4).run(reqs, clock=clk, sleep=clk.sleep)}
    assert sorted(out) == list(range(8))
    assert out[2].status == "failed" and isinstance(out[2].result, ValueError)
    assert all(out[i].status == "done" and out[i].result == i for i in out if i != 2)
    assert be.admitted == [0, 1, 3, 4, 5, 6, 7]        # admission order kept through the retries
    assert out[3].admitted >= min(out[0].finished, out[1].finished)
    assert be.in_use == 0 and be.max_in_use <= 1000
    clk2 = Clock()
    be2 = FaultyBackend(clk2, lambda r: 0.01, device_bytes=400)
    out2 = Scheduler(be2, 1500, 4).run([Request(0, 0.0, 5, 10, 10, 7, 256, 8)], clock=clk2, sleep=clk2.sleep)
    assert out2[0].status == "failed" and isinstance(out2[0].result, OutOfMemory)
