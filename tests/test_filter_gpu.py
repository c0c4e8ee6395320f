"""Sec. 3.3 light-curve outlier filter on the GPU against the FP64 oracle.

Stacks with bright interlopers planted in single epochs (the case the filter
exists for): every kept trajectory of the search is filtered on the GPU and by
the oracle.  Rejected epochs must be the same, except an epoch whose oracle
statistic |alpha_e - alpha_rest| / sigma lies within 1e-5 relative of the
threshold (the GPU reads FP32 planes, the oracle FP64 ones); the recomputed
Psi, Phi, nu and alpha must agree to 1e-5 relative (nu, alpha: with the noise
unit floors of the search's tolerance).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _compare import nu_tol
from test_parity_gpu import gpu_planes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(kb):
    c = kb.Context(0)
    yield c
    c.close()


def _with_interlopers(seed, N, H, W, n_blobs, flux):
    st = synth.small_stack(seed, N, H, W, K=5, sigma=1.0, var_lo=1.0, var_hi=2.0, nan_frac=0.01, n_angles=6,
                           n_speeds=6, s_lo=2.0, s_hi=12.0, k=4, n_sources=4, flux=25.0)
    rng = np.random.default_rng(seed + 1000)
    for _ in range(n_blobs):
        e = int(rng.integers(0, N))
        synth.render_source(st.sci[e], rng.uniform(0, W), rng.uniform(0, H), flux, 1.0, 2)
    return st


def _statistics(psi, phi, times, dxv, dyv, x0, y0):
    """Per stack epoch: the oracle's |alpha_e - alpha_rest| / sigma (nan where not tested)."""
    N, H, W = psi.shape
    P = F = 0.0
    inside = []
    for e in np.argsort(times, kind="stable"):
        x, y = x0 + dxv[e], y0 + dyv[e]
        if 0 <= x < W and 0 <= y < H:
            inside.append((e, psi[e, y, x], phi[e, y, x]))
            P += psi[e, y, x]
            F += phi[e, y, x]
    z = np.full(N, np.nan)
    for e, pe, fe in inside:
        rest = F - fe
        if fe > 0 and rest > 0:
            z[e] = abs(pe / fe - (P - pe) / rest) / math.sqrt(1 / fe + 1 / rest)
    return z


@pytest.mark.parametrize("storage,rescore", [("f32", False), ("bf16", True)])
def test_filter_matches_oracle(kb, ctx, storage, rescore):
    st = _with_interlopers(810, 8, 56, 70, n_blobs=60, flux=400.0)
    N, H, W = st.sci.shape
    s = gpu_planes(kb, ctx, st, storage)
    flags = kb.KB_RESCORE_FP64 if rescore else 0
    job = kb.Job(ctx, H, W, N, st.vx.size, st.k, flags)
    job.search(s, st.times, st.vx, st.vy, st.k, -math.inf, flags)
    res = job.results()
    filt = job.filter_lightcurves(s, 5.0)
    torch.cuda.synchronize()
    job.free()
    s.free()
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    assert np.array_equal(filt["vidx"], res["vidx"])
    n_rej = n_amb = 0
    for (y, x, i) in zip(*np.nonzero(res["vidx"] >= 0)):
        g = filt[y, x, i]
        v = int(g["vidx"])
        P, F, nk, nr, rej = oracle.filter_lightcurve(psi, phi, st.times, dx[v], dy[v], x, y, 5.0)
        grej = np.array([(g["rejected"][e >> 5] >> (e & 31)) & 1 for e in range(N)], bool)
        if not np.array_equal(grej, rej):
            z = _statistics(psi, phi, st.times, dx[v], dy[v], x, y)
            differ = np.nonzero(grej != rej)[0]
            assert np.all(np.abs(z[differ] - 5.0) <= 5e-5), (x, y, v, z[differ])
            n_amb += 1
            continue
        n_rej += nr
        assert (g["nobs"], g["nrejected"]) == (nk, nr)
        assert abs(g["psi"] - P) <= 1e-5 * (abs(P) + math.sqrt(F) + 1e-30)
        assert abs(g["phi"] - F) <= 1e-5 * F + 1e-30
        if F > 0:
            nu = P / math.sqrt(F)
            assert abs(g["nu"] - nu) <= nu_tol(nu)
            assert abs(g["alpha"] - P / F) <= 1e-5 * max(abs(P / F), 1 / math.sqrt(F))
        else:
            assert g["nu"] == -math.inf
    assert n_rej > 20, "the planted interlopers should have caused rejections"
    assert n_amb <= 2
    # a trajectory that lost an interloper epoch drops in nu; none rises above its unfiltered value
    # by more than the noise of the removed epochs (sanity of the recomputation on the GPU side)
    valid = res["vidx"] >= 0
    assert np.all(filt["nobs"][valid] + filt["nrejected"][valid] == res["nobs"][valid])


def test_filter_rejects_bad_arguments(kb, ctx):
    st = synth.small_stack(811, 3, 20, 30, K=3)
    s = gpu_planes(kb, ctx, st)
    job = kb.Job(ctx, 20, 30, 3, st.vx.size, 2)
    with pytest.raises(kb.KBError):
        job.filter_lightcurves(s, 5.0)          # no search yet
    job.search(s, st.times, st.vx, st.vy, 2)
    with pytest.raises(kb.KBError):
        job.filter_lightcurves(s, 0.0)          # nsigma must be positive
    other = gpu_planes(kb, ctx, synth.small_stack(812, 3, 21, 30, K=3))
    with pytest.raises(kb.KBError):
        job.filter_lightcurves(other, 5.0)      # not the searched stack's shape
    job.free()
    s.free()
    other.free()
