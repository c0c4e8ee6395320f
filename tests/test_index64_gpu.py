"""The search with 64-bit element offsets: stacks whose planes hold more than
2^31 elements (here 128 epochs of 4096 x 4096 in FP32, and 128 epochs of
2048 x 4096 in 16-bit storage, whose two phases double the span).

Only 4 of the 128 epochs carry data; the other 124 are masked everywhere
(infinite variance), so their psi and phi are exactly 0 and add exact zeros to
every sum.  The big stack (64-bit offsets) must therefore give the Psi, Phi, nu
and velocity of every kept trajectory of the 4-epoch stack (32-bit offsets), bit
for bit; nobs differs (it counts in-image epochs, masked or not).  The 4-epoch
search is held to the FP64 oracle on sampled start pixels.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _compare import check_topk

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = torch.device("cuda:0")
REAL = [0, 41, 87, 127]


def _records(kb, ctx, sci, var, psf, times, vx, vy, k, storage):
    N, H, W = sci.shape
    s = kb.Stack(ctx, N, H, W, storage)
    s.make_psi_phi(sci, var, None, psf)
    flags = kb.KB_RESCORE_FP64 if storage != "f32" else 0
    job = kb.Job(ctx, H, W, N, vx.size, k, flags)
    job.search(s, times, vx, vy, k, -math.inf, flags)
    out = torch.empty(H * W * k * kb.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=DEV)
    job.results(out)
    res = out.cpu().numpy().view(kb.RESULT_DTYPE).reshape(H, W, k)
    torch.cuda.synchronize()
    job.free()
    s.free()
    return res


@pytest.mark.parametrize("storage,H,W", [("f32", 4096, 4096), ("bf16", 2048, 4096)])
def test_64bit_offsets_equal_32bit_search(kb, storage, H, W):
    rng = np.random.default_rng(64)
    N, K, k = 128, 7, 4
    small = synth.small_stack(640, len(REAL), H, W, K=K, var_lo=80, var_hi=120, nan_frac=0.005,
                              times=[0.0, 0.4, 1.1, 2.0], n_angles=4, n_speeds=4, s_lo=20.0, s_hi=200.0,
                              n_sources=20, flux=60.0)
    times = np.sort(rng.uniform(0.0, 2.0, N))
    times[REAL] = small.times                      # the real epochs keep their times (t_min = 0 stays real)
    times[0] = 0.0
    psf = np.stack([small.psf[0]] * N)
    for i, e in enumerate(REAL):
        psf[e] = small.psf[i]
    sci = torch.zeros((N, H, W), dtype=torch.float32, device=DEV)
    var = torch.full((N, H, W), math.inf, dtype=torch.float32, device=DEV)
    for i, e in enumerate(REAL):
        sci[e] = torch.from_numpy(small.sci[i]).to(DEV)
        var[e] = torch.from_numpy(small.var[i]).to(DEV)
    ctx = kb.Context(0)
    big = _records(kb, ctx, sci, var, psf, times, small.vx, small.vy, k, storage)
    del sci, var
    torch.cuda.empty_cache()
    ref = _records(kb, ctx, torch.from_numpy(small.sci).to(DEV), torch.from_numpy(small.var).to(DEV), small.psf,
                   small.times, small.vx, small.vy, k, storage)
    ctx.close()
    for f in ("x0", "y0", "vidx", "vx", "vy", "psi", "phi", "nu", "alpha"):
        assert np.array_equal(big[f], ref[f]), f
    # the 4-epoch search against the oracle on sampled start pixels
    px = np.concatenate([[0, W - 1, W // 2], rng.integers(0, W, 40)])
    py = np.concatenate([[0, H - 1, H // 2], rng.integers(0, H, 40)])
    dx, dy = oracle.offsets(small.times, small.vx, small.vy)
    want = oracle.search_pixels_from_images(small.sci, small.var, None, small.psf, small.times, dx, dy, k, px, py)

    def nu_of(p, v):
        P, F, _ = oracle.trajectory_from_images(small.sci, small.var, None, small.psf, small.times, dx[v], dy[v],
                                                px[p], py[p])
        return P / math.sqrt(F) if F > 0 else -math.inf
    check_topk(ref[py, px], want, nu_of)
