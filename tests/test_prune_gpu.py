"""The thresholded search with likelihood-bound pruning (KB_PRUNE, Sec. 5.3).

Pruning skips a warp span's gathers for a velocity when the Cauchy-Schwarz bound
on nu over the span cannot reach nu_min, so its records must equal those of the
same search without the flag, byte for byte; the bound planes it builds are
compared with the oracle's (kbo_snr2_span_max, pinned by brute force), and the
thresholded search itself with the FP64 oracle.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _compare import check_topk, oracle_nu_table

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx(kb):
    c = kb.Context(0)
    yield c
    c.close()


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _stack(seed, N=6, H=70, W=300):
    return synth.small_stack(seed, N, H, W, K=5, nan_frac=0.01, mask_frac=0.01, n_angles=8, n_speeds=8, s_hi=14.0,
                             n_sources=4, flux=60.0)


def _search(kb, ctx, st, storage, k, nu_min, flags):
    N, H, W = st.sci.shape
    s = kb.Stack(ctx, N, H, W, storage)
    s.make_psi_phi(_dev(st.sci), _dev(st.var), _dev(st.mask), st.psf)
    job = kb.Job(ctx, H, W, N, st.vx.size, k, flags & kb.KB_RESCORE_FP64)
    job.search(s, st.times, st.vx, st.vy, k, nu_min, flags)
    res = job.results()
    torch.cuda.synchronize()
    return s, job, res


@pytest.mark.parametrize("storage,k", [("f32", 4), ("f32", 8), ("f32", 12), ("bf16", 8), ("f16", 8), ("f16", 12)])
@pytest.mark.parametrize("nu_min", [3.0, 4.5, 1e6])
def test_pruned_records_equal_unpruned(kb, ctx, storage, k, nu_min):
    st = _stack(500 + k)
    s0, j0, ref = _search(kb, ctx, st, storage, k, nu_min, 0)
    s1, j1, got = _search(kb, ctx, st, storage, k, nu_min, kb.KB_PRUNE)
    assert got.tobytes() == ref.tobytes()
    if nu_min < 100:
        assert (ref["vidx"] >= 0).any() and (ref["vidx"] < 0).any()   # the threshold both keeps and drops
    for o in (j0, j1, s0, s1):
        o.free()


def test_pruned_rescored_search_equals_unpruned(kb, ctx):
    st = _stack(520)
    flags = kb.KB_RESCORE_FP64
    s0, j0, ref = _search(kb, ctx, st, "bf16", 8, 3.5, flags)
    s1, j1, got = _search(kb, ctx, st, "bf16", 8, 3.5, flags | kb.KB_PRUNE)
    assert got.tobytes() == ref.tobytes()
    for o in (j0, j1, s0, s1):
        o.free()


def test_pruned_search_against_the_oracle(kb, ctx):
    st = _stack(530)
    nu_min = 4.0
    s, job, res = _search(kb, ctx, st, "f32", 8, nu_min, kb.KB_PRUNE)
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    ref = oracle.search_region(psi, phi, st.times, dx, dy, 8, nu_min)
    table = oracle_nu_table(psi, phi, st.times, dx, dy)
    check_topk(res, ref, lambda p, v: table[p, v])
    job.free()
    s.free()


@pytest.mark.parametrize("storage,span", [("f32", 64), ("bf16", 128), ("f16", 128)])
def test_bound_planes_against_the_oracle(kb, ctx, storage, span):
    """The planes the search used: entry c + span / 32 of a row is the oracle's maximum of
    max(psi, 0)^2 / phi over the columns [32 c, 32 c + span + 32) (its span maxima for windows
    span + 32 wide, at x = 32 c), over the very values the search sums (the FP32 planes, or the
    decoded 16-bit codes), rounded upwards in FP32: never below the FP64 value, and within 2^-21
    relative of it."""
    st = _stack(540)
    N, H, W = st.sci.shape
    s, job, _ = _search(kb, ctx, st, storage, 8, 3.0, kb.KB_PRUNE)
    nb, nblk = span // 32, (W + 31) // 32
    got = torch.empty(N * H * (nblk + nb), dtype=torch.float32, device=DEV)
    s.copy_planes(2, got)
    got = got.cpu().numpy().reshape(N, H, nblk + nb).astype(np.float64)
    if storage == "f32":
        pl = torch.empty((N, H, W, 2), dtype=torch.float32, device=DEV)
        s.copy_planes(0, pl)
        pl = pl.cpu().numpy().astype(np.float64)
        psi, phi = pl[..., 0], pl[..., 1]
    else:
        codes = torch.empty((N, H, W, 2), dtype=torch.int16, device=DEV)
        s.copy_planes(1, codes)
        c = codes.cpu().numpy().view(np.uint16)
        sp, sf = s.scales()
        if storage == "bf16":
            val = (c.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        else:
            val = c.view(np.float16).astype(np.float64)
        psi = val[..., 0] * sp[:, None, None]
        phi = val[..., 1] * sf[:, None, None]
    L = span + 32
    r = oracle.snr2_span_max(psi, phi, L)                  # r[..., x + L - 1]: columns [x, x + L)
    c = np.arange(-nb, nblk)
    want = r[..., 32 * c + L - 1]
    assert np.all(got >= want)
    assert np.all(got <= want * (1 + 2.0 ** -21))
    assert (want > 0).any()
    job.free()
    s.free()


def test_bound_planes_follow_new_psi_phi(kb, ctx):
    """kb_make_psi_phi on the stack invalidates its bound planes: the next pruned search rebuilds
    them and still equals the unpruned one."""
    a, b = _stack(550), _stack(551)
    N, H, W = a.sci.shape
    s = kb.Stack(ctx, N, H, W, "f32")
    job = kb.Job(ctx, H, W, N, a.vx.size, 8, 0)
    outs = []
    for st in (a, b):
        s.make_psi_phi(_dev(st.sci), _dev(st.var), _dev(st.mask), st.psf)
        for flags in (kb.KB_PRUNE, 0):
            job.search(s, st.times, st.vx, st.vy, 8, 3.5, flags)
            outs.append(job.results().tobytes())
    torch.cuda.synchronize()
    assert outs[0] == outs[1] and outs[2] == outs[3] and outs[0] != outs[2]
    job.free()
    s.free()


def test_prune_without_a_positive_threshold_is_the_plain_search(kb, ctx):
    st = _stack(560)
    s0, j0, ref = _search(kb, ctx, st, "f32", 8, -math.inf, 0)
    s1, j1, got = _search(kb, ctx, st, "f32", 8, -math.inf, kb.KB_PRUNE)
    assert got.tobytes() == ref.tobytes()
    with pytest.raises(kb.KBError):
        s1.copy_planes(2, torch.empty(1 << 20, dtype=torch.float32, device=DEV))   # none built
    for o in (j0, j1, s0, s1):
        o.free()
