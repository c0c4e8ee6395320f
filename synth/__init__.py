"""Seeded synthetic inputs for the shift-and-stack search (DECam/HiTS-shaped stand-ins).

This module only draws inputs: images, variance planes, bad-pixel masks,
Gaussian PSFs, epoch times, injected linear sources and velocity grids.  It
computes nothing of the method itself (no likelihood images, trajectory
offsets, sums or scores), so the CUDA path and the CPU oracle can both consume
it without sharing any of the method's arithmetic.

Workloads (the paper's HiTS data are replaced by synthetic stacks of the same
shape: 4K x 4K warped DECam patches, 3 nights, 4 visits per night, Sec. 3.1-3.2):

  tiny()      5 x 64 x 64, t = 0, 0.5, 1, 1.5, 2 d, N(0,1) noise, variance 1,
              7x7 Gaussian PSF (sigma 1), one source from (20.3, 30.7) at
              v = (6, -3.5) px/d with flux 8, 16 angles over [-pi, pi) x
              16 speeds over [1, 10] px/d, k = 4.
  decam()     12 x 4096 x 4096, 4 visits 1.5 h apart on each of 3 nights,
              variance per epoch U[80, 120], 1 % of pixels NaN in clusters,
              17x17 Gaussian PSF with FWHM U[3.5, 4.5] per epoch, 50 sources
              with per-epoch SNR U[1.5, 3], speeds 90-550 px/d, angles within
              +-pi/4 of +x; grid 32 angles x 32 speeds over that range, k = 8.
  batch_specs() / batch_stack() / batch_meta()
              64 uneven stacks for the batched search (W 2048 x H 4096, 5-20
              epochs over 1-4 nights, PSF sigma 1.2-2.0 px, 256-2048
              velocities, k 4-16); images_device() draws their planes on the GPU.
  serving_jobs()  the job mix of the serving loop.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

FWHM_PER_SIGMA = 2.0 * math.sqrt(2.0 * math.log(2.0))


@dataclasses.dataclass
class Stack:
    name: str
    sci: np.ndarray            # [N][H][W] float32, background-subtracted counts (NaN = bad pixel)
    var: np.ndarray            # [N][H][W] float32, variance plane
    mask: Optional[np.ndarray]  # [N][H][W] uint8 or None (non-zero = masked)
    psf: np.ndarray            # [N][K][K] float32, sums to 1
    times: np.ndarray          # [N] float64, days
    vx: np.ndarray             # [V] float64, px/day
    vy: np.ndarray             # [V] float64, px/day
    k: int                     # results kept per start pixel
    sources: list              # injected sources: dicts with x0, y0, vx, vy, flux

    @property
    def shape(self):
        return self.sci.shape


def gaussian_psf(K: int, sigma: float) -> np.ndarray:
    """K x K Gaussian sampled at integer offsets from the centre, normalised to sum 1."""
    r = K // 2
    d = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-0.5 * (d / sigma) ** 2)
    k2 = np.outer(g, g)
    return (k2 / k2.sum()).astype(np.float32)


def elliptical_psf(K: int, sigma_major: float, sigma_minor: float, theta: float) -> np.ndarray:
    """K x K elliptical Gaussian, major axis at angle theta, normalised to sum 1 (not separable
    unless the axes are equal or aligned with the grid)."""
    r = K // 2
    d = np.arange(-r, r + 1, dtype=np.float64)
    yy, xx = np.meshgrid(d, d, indexing="ij")
    c, s = math.cos(theta), math.sin(theta)
    u = c * xx + s * yy
    w = -s * xx + c * yy
    g = np.exp(-0.5 * ((u / sigma_major) ** 2 + (w / sigma_minor) ** 2))
    return (g / g.sum()).astype(np.float32)


def elongate_psfs(psf: np.ndarray, seed: int = 11, q_lo: float = 0.6, q_hi: float = 0.9) -> np.ndarray:
    """Per epoch, an elliptical version of a Gaussian PSF stack: the same major-axis width
    (its second moment), axis ratio U[q_lo, q_hi], orientation U[0, pi)."""
    rng = np.random.default_rng(seed)
    N, K = psf.shape[0], psf.shape[-1]
    r = K // 2
    d = np.arange(-r, r + 1, dtype=np.float64)
    out = []
    for e in range(N):
        sig = math.sqrt(float(np.sum(psf[e].astype(np.float64).sum(axis=0) * d ** 2)))
        out.append(elliptical_psf(K, sig, sig * rng.uniform(q_lo, q_hi), rng.uniform(0.0, math.pi)))
    return np.stack(out)


def velocity_grid(n_angles, n_speeds, theta_lo, theta_hi, s_lo, s_hi, angle_endpoint=True,
                  speed_endpoint=True):
    """Linearly spaced angle x speed grid (Sec. 3.2); index = i_angle * n_speeds + j_speed."""
    th = np.linspace(theta_lo, theta_hi, n_angles, endpoint=angle_endpoint)
    sp = np.linspace(s_lo, s_hi, n_speeds, endpoint=speed_endpoint)
    T, S = np.meshgrid(th, sp, indexing="ij")
    return (S * np.cos(T)).ravel(), (S * np.sin(T)).ravel()


def render_source(img: np.ndarray, cx: float, cy: float, flux: float, sigma: float, half: int) -> None:
    """Add a Gaussian point source centred at sub-pixel (cx, cy); pixel centres at integer indices."""
    H, W = img.shape
    ix, iy = int(math.floor(cx + 0.5)), int(math.floor(cy + 0.5))
    x_lo, x_hi = max(ix - half, 0), min(ix + half + 1, W)
    y_lo, y_hi = max(iy - half, 0), min(iy + half + 1, H)
    if x_lo >= x_hi or y_lo >= y_hi:
        return
    xs = np.arange(ix - half, ix + half + 1, dtype=np.float64)
    ys = np.arange(iy - half, iy + half + 1, dtype=np.float64)
    g = np.exp(-0.5 * ((ys[:, None] - cy) ** 2 + (xs[None, :] - cx) ** 2) / sigma ** 2)
    g /= g.sum()
    stamp = (flux * g)[y_lo - (iy - half):y_hi - (iy - half), x_lo - (ix - half):x_hi - (ix - half)]
    img[y_lo:y_hi, x_lo:x_hi] += stamp.astype(np.float32)


def nan_clusters(rng: np.random.Generator, H: int, W: int, frac: float) -> np.ndarray:
    """Boolean bad-pixel map: disks of radius 1-3 px at uniform centres until `frac` is covered."""
    bad = np.zeros((H, W), bool)
    offs = {}
    for r in (1, 2, 3):
        oy, ox = np.mgrid[-r:r + 1, -r:r + 1]
        sel = oy ** 2 + ox ** 2 <= r * r
        offs[r] = (oy[sel], ox[sel])
    target = frac * H * W
    while bad.sum() < target:
        need = target - bad.sum()
        n = max(int(need / 14.0), 1)
        radii = rng.integers(1, 4, n)
        cy = rng.integers(0, H, n)
        cx = rng.integers(0, W, n)
        for r in (1, 2, 3):
            m = radii == r
            if not m.any():
                continue
            oy, ox = offs[r]
            yy = (cy[m][:, None] + oy[None, :]).ravel()
            xx = (cx[m][:, None] + ox[None, :]).ravel()
            ok = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
            bad[yy[ok], xx[ok]] = True
    return bad


def tiny(seed: int = 0) -> Stack:
    """5 x 64 x 64 stack with one injected source (the small parity workload)."""
    rng = np.random.default_rng(seed)
    N, H, W = 5, 64, 64
    times = np.array([0.0, 0.5, 1.0, 1.5, 2.0])
    sci = rng.standard_normal((N, H, W)).astype(np.float32)
    var = np.ones((N, H, W), np.float32)
    psf = np.stack([gaussian_psf(7, 1.0)] * N)
    src = dict(x0=20.3, y0=30.7, vx=6.0, vy=-3.5, flux=8.0)
    for e in range(N):
        render_source(sci[e], src["x0"] + src["vx"] * times[e], src["y0"] + src["vy"] * times[e],
                      src["flux"], 1.0, 3)
    vx, vy = velocity_grid(16, 16, -math.pi, math.pi, 1.0, 10.0, angle_endpoint=False)
    return Stack("tiny 5x64x64", sci, var, None, psf, times, vx, vy, 4, [src])


def decam_times(nights: int = 3, visits: int = 4, cadence_h: float = 1.5) -> np.ndarray:
    return np.array([n + j * cadence_h / 24.0 for n in range(nights) for j in range(visits)])


def decam(seed: int = 1, H: int = 4096, W: int = 4096, n_sources: int = 50, n_angles: int = 32,
          n_speeds: int = 32, k: int = 8) -> Stack:
    """DECam-shaped 12-epoch stack (3 nights x 4 visits 1.5 h apart), 4096 x 4096 by default."""
    rng = np.random.default_rng(seed)
    times = decam_times()
    N = times.size
    K = 17
    var_t = rng.uniform(80.0, 120.0, N).astype(np.float32)
    fwhm = rng.uniform(3.5, 4.5, N)
    sig = fwhm / FWHM_PER_SIGMA
    psf = np.stack([gaussian_psf(K, s) for s in sig])
    sci = np.empty((N, H, W), np.float32)
    var = np.empty((N, H, W), np.float32)
    for e in range(N):
        sci[e] = rng.standard_normal((H, W), dtype=np.float32)
        sci[e] *= np.float32(math.sqrt(var_t[e]))
        var[e] = var_t[e]
    sources = []
    for _ in range(n_sources):
        snr = rng.uniform(1.5, 3.0)
        speed = rng.uniform(90.0, 550.0)
        ang = rng.uniform(-math.pi / 4, math.pi / 4)
        # flux giving a per-epoch PSF-fit SNR of `snr` for a Gaussian of effective area 4 pi sigma^2
        flux = snr * math.sqrt(4.0 * math.pi * float(np.mean(sig ** 2)) * float(np.mean(var_t)))
        s = dict(x0=rng.uniform(0, W), y0=rng.uniform(0, H), vx=speed * math.cos(ang),
                 vy=speed * math.sin(ang), flux=flux)
        sources.append(s)
        for e in range(N):
            render_source(sci[e], s["x0"] + s["vx"] * times[e], s["y0"] + s["vy"] * times[e], flux,
                          sig[e], K // 2)
    for e in range(N):
        sci[e][nan_clusters(rng, H, W, 0.01)] = np.nan
    vx, vy = velocity_grid(n_angles, n_speeds, -math.pi / 4, math.pi / 4, 90.0, 550.0)
    return Stack("decam 12x%dx%d" % (H, W), sci, var, None, psf, times, vx, vy, k, sources)


def batch_specs(seed: int = 3, count: int = 64):
    """Shapes of the uneven batch: epochs, nights, PSF sigma, grid size and k per stack."""
    rng = np.random.default_rng(seed)
    grids = [(16, 16), (32, 16), (32, 32), (64, 32)]
    specs = []
    for i in range(count):
        N = int(rng.integers(5, 21))
        nights = int(rng.integers(1, 5))
        sigma = float(rng.uniform(1.2, 2.0))
        na, ns = grids[int(rng.integers(0, 4))]
        k = int(rng.integers(4, 17))
        specs.append(dict(index=i, N=N, nights=nights, sigma=sigma, n_angles=na, n_speeds=ns, k=k,
                          seed=int(rng.integers(0, 2 ** 31))))
    return specs


def batch_times(N: int, nights: int, rng: np.random.Generator) -> np.ndarray:
    """4 visits 1.5 h apart on the first night, the remaining epochs spread over the nights."""
    t = [j * 1.5 / 24.0 for j in range(min(4, N))]
    rest = N - len(t)
    for i in range(rest):
        night = 1 + (i % max(nights - 1, 1)) if nights > 1 else 0
        t.append(night + 0.25 + rng.uniform(0.0, 0.2) + (i // max(nights - 1, 1)) * 0.0625)
    return np.sort(np.array(t))


def batch_stack(spec: dict, H: int = 4096, W: int = 2048) -> Stack:
    """One stack of the uneven batch (noise and mask model as decam())."""
    rng = np.random.default_rng(spec["seed"])
    N = spec["N"]
    times = batch_times(N, spec["nights"], rng)
    sigma = spec["sigma"]
    K = 2 * int(math.ceil(4 * sigma)) + 1
    var_t = rng.uniform(80.0, 120.0, N).astype(np.float32)
    psf = np.stack([gaussian_psf(K, sigma)] * N)
    sci = np.empty((N, H, W), np.float32)
    var = np.empty((N, H, W), np.float32)
    for e in range(N):
        sci[e] = rng.standard_normal((H, W), dtype=np.float32)
        sci[e] *= np.float32(math.sqrt(var_t[e]))
        var[e] = var_t[e]
        sci[e][nan_clusters(rng, H, W, 0.01)] = np.nan
    vx, vy = velocity_grid(spec["n_angles"], spec["n_speeds"], -math.pi / 4, math.pi / 4, 90.0, 550.0)
    return Stack("batch#%d %dx%dx%d" % (spec["index"], N, H, W), sci, var, None, psf, times, vx, vy,
                 spec["k"], [])


def batch_meta(spec: dict):
    """Host part of one batch stack: (times, psf [N][K][K], vx, vy, k), drawn as in batch_stack()."""
    rng = np.random.default_rng(spec["seed"])
    N = spec["N"]
    times = batch_times(N, spec["nights"], rng)
    K = 2 * int(math.ceil(4 * spec["sigma"])) + 1
    psf = np.stack([gaussian_psf(K, spec["sigma"])] * N)
    vx, vy = velocity_grid(spec["n_angles"], spec["n_speeds"], -math.pi / 4, math.pi / 4, 90.0, 550.0)
    return times, psf, vx, vy, spec["k"]


def images_device(seed: int, N: int, H: int, W: int, device, var_lo: float = 80.0, var_hi: float = 120.0,
                  nan_frac: float = 0.01):
    """Science and variance planes drawn on a CUDA device (torch's seeded generator), with the
    noise and bad-pixel model of decam(): per-epoch variance U[var_lo, var_hi], N(0, var) noise,
    disks of radius 1-3 px set to NaN covering about `nan_frac` of each epoch.  For workloads too
    large to draw on the host in reasonable time; returns float32 tensors [N][H][W]."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    var_t = torch.empty(N, device=device).uniform_(var_lo, var_hi, generator=g)
    sci = torch.randn((N, H, W), device=device, generator=g)
    sci *= var_t.sqrt().view(N, 1, 1)
    var = var_t.view(N, 1, 1).expand(N, H, W).contiguous()
    n = max(1, int(nan_frac * H * W / 15.67))     # mean disk area of radii 1, 2, 3: (5 + 13 + 29) / 3
    for e in range(N):
        r = torch.randint(1, 4, (n,), device=device, generator=g)
        cy = torch.randint(0, H, (n,), device=device, generator=g)
        cx = torch.randint(0, W, (n,), device=device, generator=g)
        for rad in (1, 2, 3):
            oy, ox = torch.meshgrid(torch.arange(-rad, rad + 1, device=device),
                                    torch.arange(-rad, rad + 1, device=device), indexing="ij")
            sel = oy * oy + ox * ox <= rad * rad
            oy, ox = oy[sel], ox[sel]
            m = r == rad
            yy = (cy[m][:, None] + oy[None, :]).reshape(-1)
            xx = (cx[m][:, None] + ox[None, :]).reshape(-1)
            ok = (yy >= 0) & (yy < H) & (xx >= 0) & (xx < W)
            sci[e].view(-1)[yy[ok] * W + xx[ok]] = float("nan")
    return sci, var


def serving_meta(job: dict, n_angles: int = 16):
    """Host part of one serving job: (times [N], psf [N][K][K], vx, vy, k).  Epochs as in the
    uneven batch (4 visits on the first night, the rest over 1-3 more nights), PSF sigma
    U[1.2, 2.0] px, a velocity grid of n_angles angles within +-pi/4 of +x times
    n_velocities // n_angles speeds over 90-550 px/day."""
    rng = np.random.default_rng(job["seed"])
    N = job["N"]
    times = batch_times(N, int(rng.integers(1, 5)), rng)
    sigma = float(rng.uniform(1.2, 2.0))
    K = 2 * int(math.ceil(4 * sigma)) + 1
    psf = np.stack([gaussian_psf(K, sigma)] * N)
    ns = max(1, job["n_velocities"] // n_angles)
    vx, vy = velocity_grid(n_angles, ns, -math.pi / 4, math.pi / 4, 90.0, 550.0)
    return times, psf, vx, vy, job["k"]


def serving_jobs(seed: int = 4, count: int = 2000, rate_hz: float = 1.0):
    """Job descriptions for the serving loop: Poisson arrivals, mixed sizes, epochs and grids."""
    rng = np.random.default_rng(seed)
    sizes = [(512, 512), (4096, 2048), (4096, 4096)]
    t = 0.0
    jobs = []
    for i in range(count):
        t += rng.exponential(1.0 / rate_hz)
        H, W = sizes[int(rng.integers(0, 3))]
        N = int(rng.integers(5, 16))
        nv = int(rng.integers(256, 1025))
        jobs.append(dict(index=i, arrival=t, H=H, W=W, N=N, n_velocities=nv, k=8,
                         seed=int(rng.integers(0, 2 ** 31))))
    return jobs


def small_stack(seed: int, N: int, H: int, W: int, K: int = 7, sigma: float = 1.0, var_lo: float = 1.0,
                var_hi: float = 1.0, times=None, nan_frac: float = 0.0, mask_frac: float = 0.0,
                n_angles: int = 8, n_speeds: int = 8, s_lo: float = 1.0, s_hi: float = 10.0,
                theta_lo: float = -math.pi, theta_hi: float = math.pi, k: int = 4,
                n_sources: int = 1, flux: float = 10.0) -> Stack:
    """Generic small seeded stack used by the parity and property tests."""
    rng = np.random.default_rng(seed)
    if times is None:
        times = np.sort(rng.uniform(0.0, 2.0, N))
        times[0] = 0.0
    times = np.asarray(times, np.float64)
    var_t = rng.uniform(var_lo, var_hi, N).astype(np.float32)
    sci = np.empty((N, H, W), np.float32)
    var = np.empty((N, H, W), np.float32)
    for e in range(N):
        var[e] = var_t[e] * rng.uniform(0.9, 1.1, (H, W)).astype(np.float32)
        sci[e] = rng.standard_normal((H, W), dtype=np.float32) * np.sqrt(var[e])
    psf = np.stack([gaussian_psf(K, sigma * rng.uniform(0.9, 1.1)) for _ in range(N)])
    sources = []
    for _ in range(n_sources):
        s = dict(x0=rng.uniform(0, W), y0=rng.uniform(0, H), vx=rng.uniform(-s_hi, s_hi),
                 vy=rng.uniform(-s_hi, s_hi), flux=flux)
        sources.append(s)
        for e in range(N):
            render_source(sci[e], s["x0"] + s["vx"] * times[e], s["y0"] + s["vy"] * times[e], flux, sigma,
                          K // 2)
    if nan_frac > 0:
        for e in range(N):
            sci[e][rng.random((H, W)) < nan_frac] = np.nan
    mask = None
    if mask_frac > 0:
        mask = (rng.random((N, H, W)) < mask_frac).astype(np.uint8)
    vx, vy = velocity_grid(n_angles, n_speeds, theta_lo, theta_hi, s_lo, s_hi, angle_endpoint=False)
    return Stack("small %dx%dx%d" % (N, H, W), sci, var, mask, psf, times, vx, vy, k, sources)
