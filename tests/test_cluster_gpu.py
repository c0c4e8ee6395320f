"""Sec. 3.3 DBSCAN de-duplication on the GPU against the oracle.

The reading makes every output unique (clusters labelled by their lowest core
index, border points by their nearest core neighbour, then lowest index, the
best member by nu, then lowest index), and both sides evaluate the squared
distance with the same rounded FP64 operations, so labels, core flags and the
kept candidates must be identical.  Inputs: clumps of candidates with scattered
ones and empty slots, the hand-built tie case, exact duplicates, the kept
trajectories of a real search, one all-in-one cluster and all-noise cases.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from test_oracle_pins import _clumps, _hand_clusters
from test_parity_gpu import gpu_planes
import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx(kb):
    c = kb.Context(0)
    yield c
    c.close()


def _records(kb, x0, y0, vx, vy, nu, vidx):
    rec = np.zeros(x0.size, kb.RESULT_DTYPE)
    rec["x0"], rec["y0"], rec["vx"], rec["vy"], rec["nu"], rec["vidx"] = x0, y0, vx, vy, nu, vidx
    return rec


def _compare(kb, ctx, rec, w_pos, w_vel, eps, min_samples):
    dev = torch.from_numpy(rec.view(np.uint8).copy()).to(DEV)
    label, keep, core, groups = ctx.cluster(dev, w_pos, w_vel, eps, min_samples, core=True)
    label, keep, core = label.cpu().numpy(), keep.cpu().numpy(), core.cpu().numpy()
    wl, wk, wc = oracle.cluster(rec["x0"], rec["y0"], rec["vx"], rec["vy"], rec["nu"], rec["vidx"], w_pos, w_vel,
                                eps, min_samples)
    assert np.array_equal(core, wc)
    assert np.array_equal(label, wl), np.nonzero(label != wl)[0][:10]
    assert np.array_equal(keep, wk)
    assert groups == int(wk.sum())
    return label, keep, core


@pytest.mark.parametrize("min_samples", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("w_pos,w_vel,eps", [(1.0, 0.5, 4.0), (0.5, 0.25, 2.0), (1.0, 0.05, 2.0)])
def test_cluster_matches_oracle_on_clumps(kb, ctx, min_samples, w_pos, w_vel, eps):
    rng = np.random.default_rng(int(100 * eps) + min_samples)
    rec = _records(kb, *_clumps(rng, 150, 16, 3, 4.0, 400))
    label, keep, core = _compare(kb, ctx, rec, w_pos, w_vel, eps, min_samples)
    assert keep.sum() < (rec["vidx"] >= 0).sum()
    if 3 <= min_samples <= 5:                              # border points present
        assert (~core & (rec["vidx"] >= 0) & (label != np.arange(label.size))).sum() > 0


def test_cluster_hand_example_ties(kb, ctx):
    rec = _records(kb, *_hand_clusters())
    label, keep, core = _compare(kb, ctx, rec, 1.0, 1.0, 1.0, 4)
    assert list(label) == [0, 0, 0, 0, 4, 4, 4, 4, 0, 9, -1]


def test_cluster_duplicates_and_degenerate_parameters(kb, ctx):
    rng = np.random.default_rng(7)
    x0, y0, vx, vy, nu, vidx = _clumps(rng, 40, 10, 2, 2.0, 50)
    # exact duplicates (d2 = 0) and equal nu: ties broken by index
    rec = _records(kb, np.concatenate([x0, x0[:30]]), np.concatenate([y0, y0[:30]]),
                   np.concatenate([vx, vx[:30]]), np.concatenate([vy, vy[:30]]),
                   np.concatenate([nu, nu[:30]]), np.concatenate([vidx, vidx[:30]]))
    _compare(kb, ctx, rec, 1.0, 0.5, 3.0, 3)
    # one cluster holding everything; every point its own group
    label, keep, _ = _compare(kb, ctx, rec, 1e-3, 1e-3, 100.0, 2)
    assert keep.sum() == 1
    label, keep, _ = _compare(kb, ctx, rec, 1.0, 1.0, 1e-6, 2)
    ok = rec["vidx"] >= 0
    assert keep.sum() == np.unique(np.stack([rec["x0"], rec["y0"], rec["vx"].view(np.int32),
                                             rec["vy"].view(np.int32)])[:, ok], axis=1).shape[1]
    # all empty slots
    rec2 = rec.copy()
    rec2["vidx"] = -1
    label, keep, _ = _compare(kb, ctx, rec2, 1.0, 1.0, 3.0, 2)
    assert np.all(label == -1) and not keep.any()


def test_cluster_of_search_results(kb, ctx):
    """The kept trajectories of a search around injected sources: many near-duplicates."""
    st = synth.small_stack(61, 10, 96, 128, K=5, var_lo=1.0, var_hi=1.5, nan_frac=0.01, n_angles=12, n_speeds=10,
                           s_lo=4.0, s_hi=20.0, k=8, n_sources=8, flux=30.0)
    N, H, W = st.sci.shape
    s = gpu_planes(kb, ctx, st)
    job = kb.Job(ctx, H, W, N, st.vx.size, st.k, 0)
    job.search(s, st.times, st.vx, st.vy, st.k, -math.inf, 0)
    out = torch.empty(H * W * st.k * kb.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=DEV)
    job.results(out)
    torch.cuda.synchronize()
    rec = out.cpu().numpy().view(kb.RESULT_DTYPE)
    top = np.argsort(-rec["nu"], kind="stable")[:4000]
    job.free()
    s.free()
    label, keep, core = _compare(kb, ctx, rec[np.sort(top)].copy(), 0.5, 0.2, 1.5, 4)
    assert keep.sum() < 0.5 * top.size


def test_cluster_arguments_are_checked(kb, ctx):
    rec = _records(kb, *_clumps(np.random.default_rng(3), 5, 4, 2, 1.0, 5))
    dev = torch.from_numpy(rec.view(np.uint8).copy()).to(DEV)
    for w_pos, w_vel, eps, ms in [(0.0, 1.0, 1.0, 2), (1.0, -1.0, 1.0, 2), (1.0, 1.0, 0.0, 2), (1.0, 1.0, math.nan, 2),
                                  (1.0, 1.0, 1.0, 0), (math.inf, 1.0, 1.0, 2)]:
        with pytest.raises(kb.KBError):
            ctx.cluster(dev, w_pos, w_vel, eps, ms)
    with pytest.raises(kb.KBError):                       # coordinates beyond 2^30 cells
        ctx.cluster(dev, 1.0, 1.0, 1e-12, 2)
    with pytest.raises(kb.KBError):                       # host records
        ctx.cluster(torch.from_numpy(rec.view(np.uint8).copy()), 1.0, 1.0, 1.0, 2)
    label, keep, core, groups = ctx.cluster(dev[:0], 1.0, 1.0, 1.0, 2)
    assert label.numel() == 0 and groups == 0
    # the context stays usable after the errors
    _compare(kb, ctx, rec, 1.0, 1.0, 1.0, 2)
