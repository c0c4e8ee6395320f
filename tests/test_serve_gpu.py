"""The serving loop on the GPU: each request's result is the same alone and in
the mix.

Requests of different sizes, epoch counts, velocity grids and k arrive while
others run; a budget that holds only a few of them at once forces queueing, so
requests are admitted as memory frees up and their kernels overlap on several
streams.  Every result must equal, byte for byte, the result of the same search
run alone through kb_search on the default stream (the served configuration:
BF16 planes with FP64 rescoring, and FP32).  The rescored results are also
held to the FP64 oracle.
"""
import math

import numpy as np
import pytest
import torch

import synth
from _compare import check_topk
from test_parity_gpu import oracle_search

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _requests(serve):
    rng = np.random.default_rng(21)
    shapes = [(48, 80), (64, 130), (33, 70), (96, 64), (20, 200)]
    reqs, stacks = [], []
    t = 0.0
    for i in range(12):
        H, W = shapes[i % len(shapes)]
        N = int(rng.integers(3, 9))
        st = synth.small_stack(500 + i, N, H, W, K=int(rng.choice([5, 7])), var_lo=50, var_hi=150,
                               flux=60.0, n_angles=int(rng.integers(5, 12)), n_speeds=int(rng.integers(6, 14)))
        k = int(rng.integers(2, 9))
        payload = dict(sci=torch.from_numpy(st.sci).pin_memory(), var=torch.from_numpy(st.var).pin_memory(),
                       psf=st.psf, times=st.times, vx=st.vx, vy=st.vy)
        reqs.append(serve.Request(i, t, N, H, W, st.psf.shape[-1], st.vx.size, k, payload))
        stacks.append(st)
        t += float(rng.choice([0.0, 0.002, 0.01]))
    return reqs, stacks


def _alone(kb, ctx, st, storage, flags, k):
    N, H, W = st.sci.shape
    s = kb.Stack(ctx, N, H, W, storage)
    s.make_psi_phi(torch.from_numpy(st.sci).to(DEV), torch.from_numpy(st.var).to(DEV), None, st.psf)
    job = kb.Job(ctx, H, W, N, st.vx.size, k, flags)
    job.search(s, st.times, st.vx, st.vy, k, -math.inf, flags)
    res = job.results()
    job.free()
    s.free()
    return res


@pytest.mark.parametrize("storage,rescore", [("bf16", True), ("f32", False)])
def test_each_result_same_alone_and_in_the_mix(kb, storage, rescore):
    from paper_1901_02492_gb300 import serve
    reqs, stacks = _requests(serve)
    ctx = kb.Context(0)
    be = serve.CudaBackend(ctx, DEV, storage=storage, rescore=rescore, slots=3,
                           max_npix=max(r.H * r.W for r in reqs), max_planes=max(r.N * r.H * r.W for r in reqs),
                           max_topk=8, keep_results=True)
    foot = sorted(be.estimate(r) for r in reqs)
    budget = sum(foot[-3:])                    # room for about three requests at a time
    sched = serve.Scheduler(be, budget, slots=3)
    done = sched.run(reqs)
    assert sorted(c.id for c in done) == list(range(len(reqs)))
    assert sched.peak_bytes <= budget
    assert ctx.hbm_in_use == 0                 # every stack and job released
    assert any(c.admitted > c.arrival for c in done), "the budget should have made some request wait"
    iv = be.device_intervals()
    overlap = any(a[0] < b[1] and b[0] < a[1] for i, a in enumerate(iv) for b in iv[i + 1:])
    assert overlap, "no two requests ran on the device at the same time"
    flags = kb.KB_RESCORE_FP64 if rescore else 0
    for c in done:
        r, st = reqs[c.id], stacks[c.id]
        ref = _alone(kb, ctx, st, storage, flags, r.topk)
        assert c.result.tobytes() == ref.tobytes(), "request %d differs from its search alone" % c.id
        if c.id < 3:
            oref, nu_of = oracle_search(st, k=r.topk)
            check_topk(c.result, oref, nu_of)
    ctx.close()


def test_cancelled_requests_release_their_memory(kb):
    """Cancellation on the device backend.  Every request arrives at once, one slot,
    budget for three: at the dispatch of request 0, requests 1 and 2 are resident,
    and request 1 is cancelled (released without running); request 3 is cancelled
    from its own dispatch (it runs, its result is dropped); request 6 before the run
    (it never reaches the device).  All memory is released, and the other results
    equal their searches alone."""
    from paper_1901_02492_gb300 import serve
    reqs, stacks = _requests(serve)
    for r in reqs:
        r.arrival = 0.0
    ctx = kb.Context(0)

    class Backend(serve.CudaBackend):
        def dispatch(self, h, slot):
            super().dispatch(h, slot)
            if h["r"].id == 0:
                sched.cancel(1)
            if h["r"].id == 3:
                sched.cancel(3)

    be = Backend(ctx, DEV, storage="bf16", rescore=True, slots=1,
                 max_npix=max(r.H * r.W for r in reqs), max_planes=max(r.N * r.H * r.W for r in reqs),
                 max_topk=8, keep_results=True)
    foot = sorted(be.estimate(r) for r in reqs)
    sched = serve.Scheduler(be, sum(foot[-3:]), slots=1)
    sched.cancel(6)
    done = {c.id: c for c in sched.run(reqs)}
    assert sorted(done) == list(range(len(reqs)))
    assert ctx.hbm_in_use == 0
    assert all(done[i].status == "cancelled" and done[i].result is None for i in (1, 3, 6))
    assert math.isnan(done[1].started) and not math.isnan(done[3].started) and math.isnan(done[6].admitted)
    for i, c in done.items():
        if i not in (1, 3, 6):
            assert c.status == "done"
            ref = _alone(kb, ctx, stacks[i], "bf16", kb.KB_RESCORE_FP64, reqs[i].topk)
            assert c.result.tobytes() == ref.tobytes()
    ctx.close()
