"""The allocation-free psi/phi entry point against the regular one.

kb_make_psi_phi_static is for callers that cannot allocate device memory where
they need the likelihood images (their device memory belongs to another
allocator, or their loop must not call cudaMalloc, which can block or
synchronise the device).  It keeps the PSF taps in a static device array shared
by all calls, so it is checked on two calls in a row with different stacks and
PSFs: the second call must not see the first call's taps.  It must also leave
the device's free memory unchanged.  This file is collected last on purpose.
"""
import math

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _asym(K, seed, N):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.1, 1.0, (N, K, K)).astype(np.float32)
    return (p / p.sum(axis=(1, 2), keepdims=True)).astype(np.float32)


def _regular(kb, ctx, st, bright):
    N, H, W = st.sci.shape
    s = kb.Stack(ctx, N, H, W, "f32")
    s.make_psi_phi(_dev(st.sci), _dev(st.var), _dev(st.mask), st.psf, bright)
    out = torch.empty((N, H, W, 2), dtype=torch.float32, device=DEV)
    s.copy_planes(0, out)
    torch.cuda.synchronize()
    s.free()
    return out.cpu().numpy()


def test_static_psi_phi_equals_regular_path_on_consecutive_calls(kb):
    ctx = kb.Context(0)
    cases = []
    a = synth.small_stack(301, 4, 70, 133, K=9, sigma=1.4, var_lo=50, var_hi=150, nan_frac=0.01,
                          mask_frac=0.02, flux=300.0)
    cases.append((a, math.inf))
    b = synth.small_stack(302, 3, 41, 97, K=5, var_lo=1, var_hi=3, nan_frac=0.02, flux=40.0)
    b.psf = _asym(5, 7, 3)          # not separable: the single-pass kernel and K^2 taps
    cases.append((b, 8.0))
    for st, bright in cases:
        N, H, W = st.sci.shape
        ref = _regular(kb, ctx, st, bright)
        sci, var, mask = _dev(st.sci), _dev(st.var), _dev(st.mask)
        out = torch.full((N, H, W, 2), float("nan"), dtype=torch.float32, device=DEV)
        kb.make_psi_phi_static(sci, var, mask, st.psf, out, bright)   # set-up on the first call
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info(DEV)[0]
        kb.make_psi_phi_static(sci, var, mask, st.psf, out, bright)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(DEV)[0] == free_before, "the static entry point allocated device memory"
        got = out.cpu().numpy()
        scale = np.abs(ref[..., 0]) + np.sqrt(ref[..., 1])
        assert np.all(np.abs(got[..., 0] - ref[..., 0]) <= 1e-5 * scale + 1e-30)
        assert np.all(np.abs(got[..., 1] - ref[..., 1]) <= 1e-5 * ref[..., 1] + 1e-30)
    ctx.close()


def test_static_psi_phi_rejects_more_taps_than_its_scratch(kb):
    N, H, W, K = 40, 8, 8, 63            # 40 * 2 * 63^2 floats of 2-D taps > 65536
    st = synth.small_stack(303, N, H, W, K=3)
    psf = _asym(K, 9, N)
    out = torch.empty((N, H, W, 2), dtype=torch.float32, device=DEV)
    with pytest.raises(kb.KBError) as e:
        kb.make_psi_phi_static(_dev(st.sci), _dev(st.var), None, psf, out)
    assert e.value.code == kb.KB_EINVAL
