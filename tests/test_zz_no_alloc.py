"""The allocation-free psi/phi entry point against the regular one and the oracle.

kb_make_psi_phi_static is for callers that cannot allocate device memory where
they need the likelihood images (their device memory belongs to another
allocator, or their loop must not call cudaMalloc, which can block or
synchronise the device).  It keeps the PSF taps in a static device array shared
by all calls, so it is checked on two calls in a row with different stacks and
PSFs: the second call must not see the first call's taps.  Both paths run the
same kernel on the same taps, so their planes must be equal bit for bit; both
are also compared with the FP64 oracle at the 1e-5 bar of the plane tests.  The
entry point must leave the device's free memory unchanged, refuse a capturing
stream, and the binding must refuse mismatched buffers before any launch.
This file is collected last on purpose.
"""
import math

import numpy as np
import pytest
import torch

import oracle
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


def _check_oracle(got, st, bright):
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf, None if math.isinf(bright) else bright)
    scale = np.abs(psi) + np.sqrt(phi)
    assert np.all(np.abs(got[..., 0] - psi) <= 1e-5 * scale + 1e-30)
    assert np.all(np.abs(got[..., 1] - phi) <= 1e-5 * phi + 1e-30)
    assert np.array_equal(got[..., 1] == 0, phi == 0)


def _cases():
    a = synth.small_stack(301, 4, 70, 133, K=9, sigma=1.4, var_lo=50, var_hi=150, nan_frac=0.01,
                          mask_frac=0.02, flux=300.0)
    b = synth.small_stack(302, 3, 41, 97, K=5, var_lo=1, var_hi=3, nan_frac=0.02, flux=40.0)
    b.psf = _asym(5, 7, 3)          # not separable: the single-pass kernel and K^2 taps
    return [(a, math.inf), (b, 8.0)]


def test_static_psi_phi_equals_regular_path_on_consecutive_calls(kb):
    ctx = kb.Context(0)
    for st, bright in _cases():
        N, H, W = st.sci.shape
        ref = _regular(kb, ctx, st, bright)
        sci, var, mask = _dev(st.sci), _dev(st.var), _dev(st.mask)
        out = torch.full((N, H, W, 2), float("nan"), dtype=torch.float32, device=DEV)
        kb.make_psi_phi_static(sci, var, mask, st.psf, out, bright)
        torch.cuda.synchronize()
        first = out.cpu().numpy()
        free_before = torch.cuda.mem_get_info(DEV)[0]
        out.fill_(float("nan"))
        kb.make_psi_phi_static(sci, var, mask, st.psf, out, bright)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(DEV)[0] == free_before, "the static entry point allocated device memory"
        got = out.cpu().numpy()
        # the same kernel on the same taps: identical bits, on both calls
        assert np.array_equal(first.view(np.uint32), ref.view(np.uint32))
        assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
        _check_oracle(got, st, bright)
        _check_oracle(ref, st, bright)
    ctx.close()


def test_static_psi_phi_rejects_more_taps_than_its_scratch(kb):
    N, H, W, K = 40, 8, 8, 63            # 40 * 2 * 63^2 floats of 2-D taps > 65536
    st = synth.small_stack(303, N, H, W, K=3)
    psf = _asym(K, 9, N)
    out = torch.empty((N, H, W, 2), dtype=torch.float32, device=DEV)
    with pytest.raises(kb.KBError) as e:
        kb.make_psi_phi_static(_dev(st.sci), _dev(st.var), None, psf, out)
    assert e.value.code == kb.KB_EINVAL


def test_static_psi_phi_refuses_mismatched_buffers_without_launching(kb):
    st = _cases()[0][0]
    N, H, W = st.sci.shape
    sci, var = _dev(st.sci), _dev(st.var)
    out = torch.full((N, H, W, 2), 7.0, dtype=torch.float32, device=DEV)
    bad = [
        dict(out=torch.full((N, H, W - 1, 2), 7.0, dtype=torch.float32, device=DEV)),   # out too small
        dict(sci=sci[:-1]),                                                             # fewer epochs than psf
        dict(var=var.double()),                                                         # wrong dtype
        dict(var=var.transpose(1, 2)),                                                  # not contiguous
        dict(sci=torch.from_numpy(st.sci)),                                             # host tensor
        dict(mask=torch.zeros((N, H, W), dtype=torch.float32, device=DEV)),             # mask not uint8
    ]
    for over in bad:
        kw = dict(sci=sci, var=var, mask=None, out=out)
        kw.update(over)
        with pytest.raises(ValueError):
            kb.make_psi_phi_static(kw["sci"], kw["var"], kw["mask"], st.psf, kw["out"])
        torch.cuda.synchronize()
        assert torch.all(out == 7.0) and torch.all(kw["out"] == 7.0), "a refused call wrote its output"


def test_static_psi_phi_refuses_a_capturing_stream(kb):
    st = _cases()[0][0]
    N, H, W = st.sci.shape
    sci, var = _dev(st.sci), _dev(st.var)
    out = torch.zeros((N, H, W, 2), dtype=torch.float32, device=DEV)
    x = torch.zeros(16, device=DEV)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(DEV)
    err = None
    with torch.cuda.stream(s):
        g.capture_begin()
        try:
            x.add_(1.0)
            try:
                kb.make_psi_phi_static(sci, var, None, st.psf, out, stream=s)
            except kb.KBError as e:
                err = e
        finally:
            g.capture_end()
    assert err is not None and err.code == kb.KB_EINVAL
    g.replay()
    torch.cuda.synchronize()
    assert torch.all(out == 0.0)
    # the same call outside the capture works
    kb.make_psi_phi_static(sci, var, None, st.psf, out)
    torch.cuda.synchronize()
    assert torch.isfinite(out).all() and (out[..., 1] > 0).any()
