"""Sec. 3.3 coadded postage stamps and their central moments on the GPU, against
the oracle.

Stacks in shuffled epoch order (so the search's time-order tables map back to
stack epochs), with NaN pixels, a mask and single-epoch interlopers; candidates
are kept trajectories of the search plus trajectories that run off the image
and start pixels in the corners.  Median stamps must equal the oracle's bit
for bit (the same float values are selected; the even-count average is taken
in FP64 on both sides); mean stamps sum in FP64 in time order on the GPU and
stack order in the oracle, so they may differ in the last float bit.  Moments
are held to the oracle's moments of the GPU's own stamp: FP64 sums in another
order, so m00 to 1e-12 of sum |v|, and the centred moments to 1e-9 times the
conditioning c = sum |v| / |m00| (not compared when c > 1e6, a stamp of pure
noise whose sum nearly cancels).  The cut decision must equal the one taken on
the oracle's moments with the same cuts, except where a moment lies within that
tolerance of its threshold.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from test_parity_gpu import gpu_planes

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx(kb):
    c = kb.Context(0)
    yield c
    c.close()


def _shuffled(seed, N, H, W, n_blobs=20, n_sources=3, flux=40.0):
    st = synth.small_stack(seed, N, H, W, K=5, sigma=1.0, var_lo=1.0, var_hi=2.0, nan_frac=0.02, mask_frac=0.02,
                           n_angles=6, n_speeds=6, s_lo=2.0, s_hi=12.0, k=4, n_sources=n_sources, flux=flux)
    rng = np.random.default_rng(seed + 7)
    for _ in range(n_blobs):
        synth.render_source(st.sci[int(rng.integers(0, N))], rng.uniform(0, W), rng.uniform(0, H), 300.0, 1.0, 2)
    p = rng.permutation(N)
    return synth.Stack(st.name, st.sci[p].copy(), st.var[p].copy(), None if st.mask is None else st.mask[p].copy(),
                       st.psf[p].copy(), st.times[p].copy(), st.vx, st.vy, st.k, st.sources)


def _searched(kb, ctx, st):
    N, H, W = st.sci.shape
    s = gpu_planes(kb, ctx, st)
    job = kb.Job(ctx, H, W, N, st.vx.size, st.k, 0)
    job.search(s, st.times, st.vx, st.vy, st.k, -math.inf, 0)
    res = job.results()
    s.free()
    return job, res


def _candidates(st, res, rng, n_kept=60, n_best=0):
    N, H, W = st.sci.shape
    ys, xs, ks = np.nonzero(res["vidx"] >= 0)
    pick = rng.choice(ys.size, n_kept, replace=False)
    if n_best:                                              # and the n_best highest-nu trajectories
        pick = np.concatenate([pick, np.argsort(-res["nu"][ys, xs, ks], kind="stable")[:n_best]])
    x0 = list(res["x0"][ys[pick], xs[pick], ks[pick]])
    y0 = list(res["y0"][ys[pick], xs[pick], ks[pick]])
    vi = list(res["vidx"][ys[pick], xs[pick], ks[pick]])
    # the strongest trajectory of the image, corners and edges with every velocity's extreme
    best = np.unravel_index(np.argmax(np.where(res["vidx"] >= 0, res["nu"], -np.inf)), res.shape)
    x0.append(int(res["x0"][best])), y0.append(int(res["y0"][best])), vi.append(int(res["vidx"][best]))
    fast = int(np.argmax(st.vx ** 2 + st.vy ** 2))
    for x, y in [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, 0), (0, H // 2)]:
        x0.append(x), y0.append(y), vi.append(fast)
    return np.array(x0, np.int32), np.array(y0, np.int32), np.array(vi, np.int32)


def _aperture_mask(r, aperture):
    yy, xx = np.mgrid[-r:r + 1, -r:r + 1]
    return np.ones((2 * r + 1, 2 * r + 1), bool) if aperture <= 0 else (xx * xx + yy * yy <= aperture * aperture)


def _check(kb, job, st, x0, y0, vi, r, median, cuts=None, aperture=0.0):
    N, H, W = st.sci.shape
    sci = torch.from_numpy(st.sci).to(DEV)
    mask = torch.from_numpy(st.mask).to(DEV)
    stamps, mom = job.stamps(sci, mask, x0, y0, vi, r, median=median, cuts=cuts, aperture=aperture)
    inside = _aperture_mask(r, aperture)
    stamps = stamps.cpu().numpy()
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    n_skipped = 0
    for i in range(x0.size):
        want = oracle.stamp(st.sci, st.mask, dx[vi[i]], dy[vi[i]], x0[i], y0[i], r, median=median)
        got = stamps[i]
        if median:
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32)), i
        else:
            assert np.allclose(got, want, rtol=2.0 ** -23, atol=0.0), (i, np.abs(got - want).max())
        m = oracle.moments(got, aperture)
        absum = float(np.abs(got.astype(np.float64))[inside].sum())
        assert abs(mom["m00"][i] - m[0]) <= 1e-12 * absum, (i, mom["m00"][i], m[0])
        cond = absum / abs(m[0]) if m[0] != 0 else math.inf
        if cond > 1e6:
            n_skipped += 1
            continue
        tol = 1e-9 * cond
        for name, w in zip(("mx", "my", "mu20", "mu02", "mu11"), m[1:]):
            assert abs(mom[name][i] - w) <= tol * max(abs(w), 1.0), (i, name, mom[name][i], w)
        if cuts is None:
            assert mom["passed"][i] == 1
            continue
        m00, mx, my, mu20, mu02, mu11 = m
        edges = [abs(mx) - cuts["max_offset"], abs(my) - cuts["max_offset"], mu20 - cuts["min_var"],
                 mu20 - cuts["max_var"], mu02 - cuts["min_var"], mu02 - cuts["max_var"],
                 abs(mu11) - cuts["max_mu11"]]
        if min(abs(e) for e in edges) <= 2 * tol * max(1.0, abs(mu20), abs(mu02)):
            continue
        want_pass = (m00 > 0 and abs(mx) <= cuts["max_offset"] and abs(my) <= cuts["max_offset"]
                     and cuts["min_var"] <= mu20 <= cuts["max_var"] and cuts["min_var"] <= mu02 <= cuts["max_var"]
                     and abs(mu11) <= cuts["max_mu11"])
        assert mom["passed"][i] == int(want_pass), (i, m)
    assert n_skipped <= x0.size // 4
    return stamps, mom


@pytest.mark.parametrize("r", [0, 3, 10, 15])
@pytest.mark.parametrize("median", [False, True])
@pytest.mark.parametrize("aperture", [0.0, 3.0])
def test_stamps_match_oracle(kb, ctx, r, median, aperture):
    st = _shuffled(900 + r, 9, 48, 61)
    job, res = _searched(kb, ctx, st)
    x0, y0, vi = _candidates(st, res, np.random.default_rng(r))
    _check(kb, job, st, x0, y0, vi, r, median, aperture=aperture)
    job.free()


def test_median_with_the_maximum_epoch_count(kb, ctx):
    """128 epochs: the per-thread selection at its full length, odd and even counts."""
    st = _shuffled(931, 128, 24, 30, n_blobs=100)
    job, res = _searched(kb, ctx, st)
    x0, y0, vi = _candidates(st, res, np.random.default_rng(1), n_kept=20)
    stamps, _ = _check(kb, job, st, x0, y0, vi, 4, True)
    job.free()
    assert np.any(stamps != 0)


def test_moment_cuts(kb, ctx):
    """The moment filter on stamps of bright sources (PSF-like: they pass), of noise and of
    interlopers: the decision equals the one taken on the oracle's moments with the same cuts."""
    st = _shuffled(944, 12, 64, 64, n_blobs=40, n_sources=6, flux=200.0)
    job, res = _searched(kb, ctx, st)
    x0, y0, vi = _candidates(st, res, np.random.default_rng(2), n_kept=100, n_best=40)
    cuts = {"max_offset": 1.0, "min_var": 0.25, "max_var": 4.0, "max_mu11": 1.0}
    _, mom = _check(kb, job, st, x0, y0, vi, 5, True, cuts=cuts)
    assert 0 < int(mom["passed"].sum()) < mom.size
    _, mom = _check(kb, job, st, x0, y0, vi, 8, False, cuts=cuts, aperture=3.0)
    assert 0 < int(mom["passed"].sum()) < mom.size
    job.free()


def test_stamp_arguments_are_checked(kb, ctx):
    st = _shuffled(950, 5, 16, 20)
    N, H, W = st.sci.shape
    sci = torch.from_numpy(st.sci).to(DEV)
    fresh = kb.Job(ctx, H, W, N, st.vx.size, st.k, 0)
    with pytest.raises(kb.KBError):                         # no search yet
        fresh.stamps(sci, None, [0], [0], [0], 2)
    fresh.free()
    job, _ = _searched(kb, ctx, st)
    for args in [([W], [0], [0], 2), ([0], [H], [0], 2), ([0], [0], [st.vx.size], 2), ([0], [0], [0], 16),
                 ([-1], [0], [0], 2)]:
        with pytest.raises(kb.KBError):
            job.stamps(sci, None, *args)
    with pytest.raises(kb.KBError):                         # not the searched stack's shape
        job.stamps(sci[:, :, :W - 1].contiguous(), None, [0], [0], [0], 2)
    with pytest.raises(kb.KBError):                         # host images
        job.stamps(torch.from_numpy(st.sci), None, [0], [0], [0], 2)
    empty, mom = job.stamps(sci, None, [], [], [], 3)
    assert empty.shape == (0, 7, 7) and mom.size == 0
    job.free()
