"""The batched search (one persistent, graph-captured launch per group of searches
with the same storage and list length) against the one-search path and the oracle.

Each search of a batch must give the records that kb_search gives for the same
arguments and the same tile shape, byte for byte: the batch kernel runs the same
tile body, only the assignment of tiles to CTAs differs.  The stacks differ in
size, epoch count, velocity grid, k, storage and rescoring, as in the uneven
batch workload, at sizes the oracle checks in seconds.
"""
import math

import numpy as np
import pytest
import torch

import synth
from _compare import check_topk
from test_parity_gpu import gpu_planes, oracle_search

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(kb):
    c = kb.Context(0)
    yield c
    c.close()


def _uneven_cases():
    """(stack, storage, k, flags) with ragged sizes, 3-14 epochs and 60-400 velocities."""
    rng = np.random.default_rng(11)
    cases = []
    shapes = [(5, 70, 133), (9, 64, 200), (3, 41, 97), (14, 33, 150), (7, 96, 64), (6, 17, 300)]
    storages = ["f32", "bf16", "f32", "f16", "f32", "bf16"]
    for i, ((N, H, W), sto) in enumerate(zip(shapes, storages)):
        st = synth.small_stack(400 + i, N, H, W, K=int(rng.choice([5, 7, 9])), nan_frac=0.01, mask_frac=0.01,
                               flux=30.0, n_angles=int(rng.integers(6, 20)), n_speeds=int(rng.integers(10, 20)))
        k = int(rng.integers(1, 17))
        flags = 1 if sto != "f32" or i == 2 else 0   # 16-bit storage with FP64 rescoring; one FP32 too
        cases.append((st, sto, k, flags))
    return cases


def _kkeep(k, flags, storage):
    """Candidates the search kernel keeps per pixel: k, plus the rescoring margin."""
    if not flags:
        return k
    return k + (max(2, k // 2) if storage == "bf16" else max(2, k // 4))


def _single(kb, ctx, stacks, cases, variant):
    ctx.set_search_variant(variant)
    out = []
    for s, (st, sto, k, flags) in zip(stacks, cases):
        N, H, W = st.sci.shape
        job = kb.Job(ctx, H, W, N, len(st.vx), k, flags)
        job.search(s, st.times, st.vx, st.vy, k, -math.inf, flags)
        out.append(job.results())
        job.free()
    ctx.set_search_variant(0)
    return out


def _batched(kb, ctx, stacks, cases, autotune, runs=1):
    jobs, searches = [], []
    for s, (st, sto, k, flags) in zip(stacks, cases):
        N, H, W = st.sci.shape
        job = kb.Job(ctx, H, W, N, len(st.vx), k, flags)
        jobs.append(job)
        searches.append(dict(job=job, stack=s, times=st.times, vx=st.vx, vy=st.vy, topk=k, flags=flags))
    b = kb.Batch(ctx, searches, autotune=autotune)
    for _ in range(runs):
        b.run()
    res = [j.results() for j in jobs]
    groups = b.groups()
    b.free()
    for j in jobs:
        j.free()
    return res, groups


@pytest.fixture(scope="module")
def uneven(kb, ctx):
    cases = _uneven_cases()
    stacks = [gpu_planes(kb, ctx, st, sto) for (st, sto, k, flags) in cases]
    torch.cuda.synchronize()
    yield cases, stacks
    for s in stacks:
        s.free()


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_batch_equals_single_searches_per_shape(kb, ctx, uneven, variant):
    cases, stacks = uneven
    ref = _single(kb, ctx, stacks, cases, variant)
    ctx.set_search_variant(variant)
    got, groups = _batched(kb, ctx, stacks, cases, autotune=False, runs=2)   # replayed graph
    ctx.set_search_variant(0)
    assert sorted(set(g.storage for g in groups)) == [0, 1, 2]
    assert all(g.variant == variant and g.index_bits == 32 for g in groups)
    assert len({(g.storage, g.kmax) for g in groups}) == len(groups)
    for i, (a, b) in enumerate(zip(got, ref)):
        assert a.shape == b.shape
        assert a.tobytes() == b.tobytes(), "search %d of the batch differs from kb_search" % i


def test_autotuned_batch_matches_single_searches_and_oracle(kb, ctx, uneven):
    cases, stacks = uneven
    got, groups = _batched(kb, ctx, stacks, cases, autotune=True)
    for g in groups:
        assert 1 <= g.variant <= 4 and g.schedule in (0, 1)
        assert all(g.tuned_ms[v] > 0 and g.tuned_ms_launch[v] > 0 for v in range(1, 5))
        chosen = (g.tuned_ms_launch if g.schedule else g.tuned_ms)[g.variant]
        assert chosen == min(min(g.tuned_ms[1:5]), min(g.tuned_ms_launch[1:5]))
        assert g.n_items > 0 and g.evals > 0
    shape_of = {(g.storage, g.kmax): g.variant for g in groups}
    names = {"f32": 0, "bf16": 1, "f16": 2}
    for i, ((st, sto, k, flags), s) in enumerate(zip(cases, stacks)):
        ref = _single(kb, ctx, [s], [(st, sto, k, flags)], shape_of[(names[sto], _kkeep(k, flags, sto))])[0]
        assert got[i].tobytes() == ref.tobytes(), "search %d differs from kb_search with the tuned shape" % i
        if sto == "f32" and not flags:
            oref, nu_of = oracle_search(st, k=k)
            check_topk(got[i], oref, nu_of)


def test_batch_rejects_shared_and_busy_jobs(kb, ctx, uneven):
    cases, stacks = uneven
    st, sto, k, flags = cases[0]
    N, H, W = st.sci.shape
    job = kb.Job(ctx, H, W, N, len(st.vx), k, 0)
    d = dict(job=job, stack=stacks[0], times=st.times, vx=st.vx, vy=st.vy, topk=k)
    with pytest.raises(kb.KBError) as e:
        kb.Batch(ctx, [d, dict(d)], autotune=False)
    assert e.value.code == kb.KB_EINVAL and "share a job" in str(e.value)
    b = kb.Batch(ctx, [d], autotune=False)
    with pytest.raises(kb.KBError) as e:          # the job's tables belong to the batch
        job.search(stacks[0], st.times, st.vx, st.vy, k)
    assert e.value.code == kb.KB_EINVAL
    with pytest.raises(kb.KBError):
        kb.Batch(ctx, [d], autotune=False)
    bad = dict(d, topk=k + 17)                    # an item failing kb_search's checks names itself
    job2 = kb.Job(ctx, H, W, N, len(st.vx), k, 0)
    with pytest.raises(kb.KBError) as e:
        kb.Batch(ctx, [dict(bad, job=job2)], autotune=False)
    assert "item 0" in str(e.value)
    b.free()
    job.search(stacks[0], st.times, st.vx, st.vy, k)   # released by kb_batch_free
    job.wait()
    job.free()
    job2.free()


def test_batch_reruns_after_planes_change(kb, ctx):
    """The graph reads the stacks' planes at run time: new psi/phi, same batch, new results."""
    a = synth.small_stack(420, 5, 40, 90, K=5, flux=30.0)
    b = synth.small_stack(421, 5, 40, 90, K=5, flux=30.0)
    s = gpu_planes(kb, ctx, a, "f32")
    job = kb.Job(ctx, 40, 90, 5, len(a.vx), 4, 0)
    bt = kb.Batch(ctx, [dict(job=job, stack=s, times=a.times, vx=a.vx, vy=a.vy, topk=4)], autotune=False)
    bt.run()
    r1 = job.results()
    from test_parity_gpu import to_dev
    s.make_psi_phi(to_dev(b.sci), to_dev(b.var), to_dev(b.mask), b.psf)
    bt.run()
    r2 = job.results()
    bt.free()
    job.free()
    s.free()
    o1, nu1 = oracle_search(a, k=4)
    b2 = synth.Stack(b.name, b.sci, b.var, b.mask, b.psf, a.times, a.vx, a.vy, 4, [])
    o2, nu2 = oracle_search(b2, k=4)
    check_topk(r1, o1, nu1)
    check_topk(r2, o2, nu2)
