"""Reduced-precision search: 16-bit psi/phi storage with per-epoch power-of-two
scales, FP32 accumulation, and FP64 rescoring of the kept candidates.

Without rescoring, nu of every kept trajectory must lie within a bound derived
from the storage format's unit roundoff u (bf16 2^-8, fp16 2^-11):
    |dPsi| <= u sum_t |psi_t| + N 2^-24 sum_t |psi_t| + N s_psi 2^-25   (fp16 subnormals)
    |dPhi| <= u sum_t  phi_t  + N 2^-24 sum_t  phi_t
    |dnu|  <= |dPsi| / sqrt(Phi) + |Psi| |dPhi| / (2 Phi^1.5)  (+ 1e-5 |nu| for the FP32 planes)
With rescoring, the top-k must match the FP64 oracle like the FP32 path
(nu within 1e-5 relative, identical lists up to near-ties).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _compare import check_topk, oracle_nu_table
from test_parity_gpu import DEV, gpu_planes, gpu_search, oracle_search, to_dev

pytestmark = pytest.mark.gpu
UNIT = {"bf16": 2.0 ** -8, "f16": 2.0 ** -11}


@pytest.fixture(scope="module")
def ctx(kb):
    c = kb.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def stack16():
    return synth.small_stack(21, 6, 96, 200, K=9, sigma=1.5, var_lo=80, var_hi=120, nan_frac=0.01,
                             n_angles=8, n_speeds=8, s_hi=15.0, k=8, n_sources=4, flux=120.0)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_codes_and_scales(kb, ctx, stack16, storage):
    st = stack16
    N, H, W = st.sci.shape
    s = gpu_planes(kb, ctx, st, storage)
    f32 = torch.empty((N, H, W, 2), dtype=torch.float32, device=DEV)
    q = torch.empty((N, H, W, 2), dtype=torch.int16, device=DEV)
    s.copy_planes(0, f32)
    s.copy_planes(1, q)
    sp, sf = s.scales()
    f = f32.cpu().numpy()
    dt = torch.bfloat16 if storage == "bf16" else torch.float16
    vals = q.view(dt).float().cpu().numpy()
    for e in range(N):
        for c, sc in ((0, sp[e]), (1, sf[e])):
            assert sc > 0 and math.frexp(float(sc))[0] == 0.5          # a power of two
            m = np.abs(f[e, ..., c]).max()
            assert 2.0 ** 14 <= m / sc < 2.0 ** 15                      # largest code in [2^14, 2^15)
            err = np.abs(vals[e, ..., c] * sc - f[e, ..., c])
            assert np.all(err <= UNIT[storage] * np.abs(f[e, ..., c]) + sc * 2.0 ** -24)
    s.free()


def _bound(storage, st, dx, dy, psi, phi, px, py, vidx, sp):
    """Per-trajectory nu error bound of the 16-bit search (see module docstring)."""
    u = UNIT[storage]
    N, H, W = psi.shape
    out = np.empty(px.size)
    for i in range(px.size):
        ap = af = P = F = 0.0
        for e in range(N):
            x, y = px[i] + dx[vidx[i], e], py[i] + dy[vidx[i], e]
            if 0 <= x < W and 0 <= y < H:
                ap += abs(psi[e, y, x])
                af += phi[e, y, x]
                P += psi[e, y, x]
                F += phi[e, y, x]
        dP = (u + N * 2.0 ** -24) * ap + (N * float(sp.max()) * 2.0 ** -25 if storage == "f16" else 0.0)
        dF = (u + N * 2.0 ** -24) * af
        out[i] = 1.01 * (dP / math.sqrt(F) + abs(P) * dF / (2.0 * F ** 1.5)) + 1e-5 * max(abs(P / math.sqrt(F)), 1)
    return out


@pytest.mark.parametrize("storage", ["bf16", "f16"])
def test_16bit_search_within_bound(kb, ctx, stack16, storage):
    st = stack16
    N, H, W = st.sci.shape
    res = gpu_search(kb, ctx, st, storage)
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    s = gpu_planes(kb, ctx, st, storage)
    sp, _ = s.scales()
    s.free()
    rng = np.random.default_rng(3)
    sel = rng.choice(H * W, 400, replace=False)
    flat = res.reshape(H * W, -1)[sel]
    py, px = np.divmod(sel, W)
    py = np.repeat(py, st.k)
    px = np.repeat(px, st.k)
    v = flat["vidx"].ravel()
    ok = v >= 0
    bound = _bound(storage, st, dx, dy, psi, phi, px[ok], py[ok], v[ok], sp)
    nu_true = np.empty(ok.sum())
    for i, (x, y, vv) in enumerate(zip(px[ok], py[ok], v[ok])):
        P = F = 0.0
        for e in range(N):
            xx, yy = x + dx[vv, e], y + dy[vv, e]
            if 0 <= xx < W and 0 <= yy < H:
                P += psi[e, yy, xx]
                F += phi[e, yy, xx]
        nu_true[i] = P / math.sqrt(F)
    err = np.abs(flat["nu"].ravel()[ok] - nu_true)
    assert np.all(err <= bound), "max excess %.3g" % (err - bound).max()
    rel = err / np.maximum(np.abs(nu_true), 1.0)
    print("%s search: max nu error %.3g (relative to max(|nu|,1)), mean %.3g" % (storage, rel.max(), rel.mean()))


@pytest.mark.parametrize("storage", ["bf16", "f16", "f32"])
def test_rescored_matches_fp64_oracle(kb, ctx, stack16, storage):
    st = stack16
    res = gpu_search(kb, ctx, st, storage, flags=kb.KB_RESCORE_FP64)
    ref, nu_of = oracle_search(st)
    check_topk(res, ref, nu_of)
    valid = ref["vidx"] >= 0
    rel = np.abs(res["nu"][valid] - ref["nu"][valid]) / np.maximum(np.abs(ref["nu"][valid]), 1.0)
    assert rel.max() <= 1e-5
    print("%s + FP64 rescoring: max nu error vs oracle %.3g" % (storage, rel.max()))


def test_rescored_tiny_and_k16(kb, ctx):
    st = synth.tiny()
    for storage in ("bf16", "f16"):
        res = gpu_search(kb, ctx, st, storage, flags=kb.KB_RESCORE_FP64)
        ref, nu_of = oracle_search(st)
        check_topk(res, ref, nu_of)
    st2 = synth.small_stack(22, 5, 40, 70, K=7, n_angles=8, n_speeds=4, k=16)
    res = gpu_search(kb, ctx, st2, "bf16", k=16, flags=kb.KB_RESCORE_FP64)
    ref, nu_of = oracle_search(st2, k=16)
    check_topk(res, ref, nu_of)


@pytest.mark.parametrize("storage", ["bf16", "f16", "f32"])
def test_key_lists_rescore_like_value_lists(kb, ctx, stack16, storage):
    """The automatic shape keeps the rescoring's candidate lists as 32-bit keys (nu rounded
    upwards in the key's high bits, the velocity index in its low bits); the value-list shape
    (variant 1 for 16-bit storage, 2 for FP32) keeps the nu of the search.  Both end in the
    exact FP64 top-k, so their rescored records must be the same bytes."""
    st = stack16
    N, H, W = st.sci.shape
    out = []
    for variant in (0, 2 if storage == "f32" else 1):
        ctx.set_search_variant(variant)
        try:
            s = gpu_planes(kb, ctx, st, storage)
            job = kb.Job(ctx, H, W, N, st.vx.size, st.k, kb.KB_RESCORE_FP64)
            job.search(s, st.times, st.vx, st.vy, st.k, -math.inf, kb.KB_RESCORE_FP64)
            out.append((job.results().tobytes(), job.repaired()))
            torch.cuda.synchronize()
            job.free()
            s.free()
        finally:
            ctx.set_search_variant(0)
    assert out[0][0] == out[1][0]
    print("%s: repaired pixels, key lists %d, value lists %d" % (storage, out[0][1], out[1][1]))
