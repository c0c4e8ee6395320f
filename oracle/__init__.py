"""FP64 CPU oracle for the shift-and-stack likelihood search (arXiv:1901.02492).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only callers.  The arithmetic lives in ``kb_oracle.c``
(plain C, FP64, no code shared with the CUDA library); this module compiles it
with gcc and marshals numpy arrays through ctypes.

Functions and the paper passages they follow:
  psi_phi            Sec. 2.1.5, the Psi/Phi likelihood images (direct 2-D correlation)
  psi_phi_at         the same definition at one pixel
  offsets            Sec. 2.2 trajectory pixels y0 + v t (fixed-point round-half-up)
  sums_one_velocity  Sec. 2.1.5 coadd Psi = sum_t psi_t(y_t), Phi = sum_t phi_t(y_t)
  search_region / search_pixels
                     Sec. 2.2 exhaustive search, scores of Sec. 2.1.5, top-k per pixel
  trajectory_from_images / search_pixels_from_images
                     one trajectory / the search at listed pixels straight from the raw
                     images (sampled checks of full-size runs)
"""
from __future__ import annotations

import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kb_oracle.c")
_LIB = os.path.join(_HERE, "libkb_oracle.so")
_lock = threading.Lock()
_lib = None

REC_DTYPE = np.dtype([("x0", "<i4"), ("y0", "<i4"), ("vidx", "<i4"), ("nobs", "<i4"),
                      ("psi", "<f8"), ("phi", "<f8"), ("nu", "<f8"), ("alpha", "<f8")])


_CMD = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off"]


def _digest() -> str:
    """sha256 of the source and the compiler command (not file times, which a copied
    tree does not keep in order)."""
    h = hashlib.sha256(" ".join(_CMD).encode())
    with open(_SRC, "rb") as f:
        h.update(f.read())
    return h.hexdigest()


def build(force: bool = False) -> str:
    """Compile kb_oracle.c into libkb_oracle.so (gcc, OpenMP, no FP contraction)."""
    stamp = _LIB + ".sha256"
    digest = _digest()
    if not force and os.path.exists(_LIB) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    subprocess.run(_CMD + ["-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    with open(stamp + ".tmp%d" % os.getpid(), "w") as f:
        f.write(digest + "\n")
    os.replace(stamp + ".tmp%d" % os.getpid(), stamp)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i32, i64, f64 = ctypes.c_int, ctypes.c_int64, ctypes.c_double
            lib.kbo_psi_phi.argtypes = [P, P, P, P, i32, i32, i32, i32, f64, P, P]
            lib.kbo_psi_phi_at.argtypes = [P, P, P, P, i32, i32, i32, f64, i32, i32, P, P]
            lib.kbo_offsets.argtypes = [P, i32, P, P, i32, P, P]
            lib.kbo_quant_velocity.argtypes = [f64]
            lib.kbo_quant_velocity.restype = i64
            lib.kbo_quant_time.argtypes = [f64]
            lib.kbo_quant_time.restype = i64
            lib.kbo_offset.argtypes = [i64, i64]
            lib.kbo_offset.restype = i64
            lib.kbo_sums_one_velocity.argtypes = [P, P, P, i32, i32, i32, P, P, P, P, P]
            lib.kbo_filter_lightcurve.argtypes = [P, P, P, i32, i32, i32, P, P, i32, i32, f64, P, P, P, P, P]
            lib.kbo_stamp.argtypes = [P, P, i32, i32, i32, P, P, i32, i32, i32, i32, P]
            lib.kbo_moments.argtypes = [P, i32, f64, P, P, P, P, P, P]
            lib.kbo_cluster.argtypes = [P, P, P, P, P, P, ctypes.c_long, f64, f64, f64, i32, P, P, P]
            lib.kbo_snr2_span_max.argtypes = [P, P, i32, i32, i32, i32, P]
            lib.kbo_span_bound.argtypes = [P, i32, i32, i32, i32, P, P, i32, i32]
            lib.kbo_span_bound.restype = f64
            lib.kbo_search_pixels.argtypes = [P, P, P, i32, i32, i32, P, P, i32, i32, f64, P, P, i64, P]
            lib.kbo_search_region.argtypes = [P, P, P, i32, i32, i32, P, P, i32, i32, f64,
                                              i32, i32, i32, i32, P]
            lib.kbo_trajectory_from_images.argtypes = [P, P, P, P, P, i32, i32, i32, i32, f64,
                                                       P, P, i32, i32, P, P, P]
            lib.kbo_search_pixels_from_images.argtypes = [P, P, P, P, P, i32, i32, i32, i32, f64, P, P, i32,
                                                          i32, f64, P, P, i64, P]
            lib.kbo_num_threads.restype = i32
            lib.kbo_set_num_threads.argtypes = [i32]
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return _load().kbo_num_threads()


def set_num_threads(n: int) -> None:
    _load().kbo_set_num_threads(int(n))


def _bright(bright_max):
    return float("inf") if bright_max is None else float(bright_max)


def psi_phi(sci, var, mask, psf, bright_max=None):
    """psi, phi planes [N][H][W] (float64) from sci/var [N][H][W] float32, mask u8 or None,
    psf [N][K][K] float32."""
    lib = _load()
    sci = _c(sci, np.float32)
    var = _c(var, np.float32)
    mask = None if mask is None else _c(mask, np.uint8)
    psf = _c(psf, np.float32)
    N, H, W = sci.shape
    K = psf.shape[-1]
    assert psf.shape == (N, K, K) and K % 2 == 1
    psi = np.empty((N, H, W), np.float64)
    phi = np.empty((N, H, W), np.float64)
    lib.kbo_psi_phi(_ptr(sci), _ptr(var), _ptr(mask), _ptr(psf), N, H, W, K, _bright(bright_max),
                    _ptr(psi), _ptr(phi))
    return psi, phi


def psi_phi_at(sci_t, var_t, mask_t, psf_t, x, y, bright_max=None):
    """psi, phi of one epoch ([H][W] inputs, [K][K] psf) at pixel (x, y)."""
    lib = _load()
    sci_t = _c(sci_t, np.float32)
    var_t = _c(var_t, np.float32)
    mask_t = None if mask_t is None else _c(mask_t, np.uint8)
    psf_t = _c(psf_t, np.float32)
    H, W = sci_t.shape
    K = psf_t.shape[-1]
    a = ctypes.c_double()
    b = ctypes.c_double()
    lib.kbo_psi_phi_at(_ptr(sci_t), _ptr(var_t), _ptr(mask_t), _ptr(psf_t), H, W, K, _bright(bright_max),
                       int(x), int(y), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def quant_velocity(v: float) -> int:
    return _load().kbo_quant_velocity(float(v))


def quant_time(dt: float) -> int:
    return _load().kbo_quant_time(float(dt))


def offset(vq: int, tq: int) -> int:
    return _load().kbo_offset(int(vq), int(tq))


def offsets(times, vx, vy):
    """dx, dy int32 [V][N] for the caller's epoch order."""
    lib = _load()
    times = _c(times, np.float64)
    vx = _c(vx, np.float64)
    vy = _c(vy, np.float64)
    N, V = times.size, vx.size
    dx = np.empty((V, N), np.int32)
    dy = np.empty((V, N), np.int32)
    lib.kbo_offsets(_ptr(times), N, _ptr(vx), _ptr(vy), V, _ptr(dx), _ptr(dy))
    return dx, dy


def sums_one_velocity(psi, phi, times, dx_v, dy_v):
    """Psi, Phi (float64) and nobs (int32) maps [H][W] for one velocity's offsets [N]."""
    lib = _load()
    psi = _c(psi, np.float64)
    phi = _c(phi, np.float64)
    times = _c(times, np.float64)
    dx_v = _c(dx_v, np.int32)
    dy_v = _c(dy_v, np.int32)
    N, H, W = psi.shape
    P = np.empty((H, W), np.float64)
    F = np.empty((H, W), np.float64)
    n = np.empty((H, W), np.int32)
    lib.kbo_sums_one_velocity(_ptr(psi), _ptr(phi), _ptr(times), N, H, W, _ptr(dx_v), _ptr(dy_v),
                              _ptr(P), _ptr(F), _ptr(n))
    return P, F, n


def filter_lightcurve(psi, phi, times, dx_v, dy_v, x0, y0, nsigma=5.0):
    """Sec. 3.3 outlier filter of one trajectory: (Psi, Phi, nkept, nrejected, rejected[N] bool)
    over the kept epochs (see kbo_filter_lightcurve for the reading)."""
    lib = _load()
    psi = _c(psi, np.float64)
    phi = _c(phi, np.float64)
    times = _c(times, np.float64)
    dx_v = _c(dx_v, np.int32)
    dy_v = _c(dy_v, np.int32)
    N, H, W = psi.shape
    P, F = ctypes.c_double(), ctypes.c_double()
    nk, nr = ctypes.c_int32(), ctypes.c_int32()
    rej = np.zeros(N, np.uint8)
    lib.kbo_filter_lightcurve(_ptr(psi), _ptr(phi), _ptr(times), N, H, W, _ptr(dx_v), _ptr(dy_v), int(x0), int(y0),
                              float(nsigma), ctypes.byref(P), ctypes.byref(F), ctypes.byref(nk), ctypes.byref(nr),
                              _ptr(rej))
    return P.value, F.value, nk.value, nr.value, rej.astype(bool)


def stamp(sci, mask, dx_v, dy_v, x0, y0, r, median=False):
    """Sec. 3.3 coadded postage stamp [2r+1][2r+1] (float32) of one trajectory: the mean or
    median over epochs of the finite, unmasked, in-image science pixels."""
    lib = _load()
    sci = _c(sci, np.float32)
    mask = None if mask is None else _c(mask, np.uint8)
    dx_v = _c(dx_v, np.int32)
    dy_v = _c(dy_v, np.int32)
    N, H, W = sci.shape
    out = np.empty((2 * r + 1, 2 * r + 1), np.float32)
    lib.kbo_stamp(_ptr(sci), None if mask is None else _ptr(mask), N, H, W, _ptr(dx_v), _ptr(dy_v), int(x0), int(y0),
                  int(r), 1 if median else 0, _ptr(out))
    return out


def moments(st, aperture=0.0):
    """(m00, mx, my, mu20, mu02, mu11) of a stamp over the central aperture x^2 + y^2 <=
    aperture^2 (the whole stamp when aperture <= 0), coordinates relative to its centre."""
    lib = _load()
    st = _c(st, np.float32)
    r = (st.shape[0] - 1) // 2
    vals = [ctypes.c_double() for _ in range(6)]
    lib.kbo_moments(_ptr(st), r, float(aperture), *[ctypes.byref(v) for v in vals])
    return tuple(v.value for v in vals)


def cluster(x0, y0, vx, vy, nu, vidx, w_pos, w_vel, eps, min_samples):
    """Sec. 3.3 DBSCAN de-duplication (reading in kb_oracle.c): (label int32, keep bool, core bool)
    per candidate.  label: the group's lowest core index, a noise point's own index, -1 for vidx < 0."""
    lib = _load()
    x0 = _c(x0, np.int32)
    y0 = _c(y0, np.int32)
    vx = _c(vx, np.float32)
    vy = _c(vy, np.float32)
    nu = _c(nu, np.float64)
    vidx = _c(vidx, np.int32)
    n = x0.size
    label = np.empty(n, np.int32)
    keep = np.empty(n, np.uint8)
    core = np.empty(n, np.uint8)
    lib.kbo_cluster(_ptr(x0), _ptr(y0), _ptr(vx), _ptr(vy), _ptr(nu), _ptr(vidx), n, float(w_pos), float(w_vel),
                    float(eps), int(min_samples), _ptr(label), _ptr(keep), _ptr(core))
    return label, keep.astype(bool), core.astype(bool)


def snr2_span_max(psi, phi, span):
    """Sec. 5.3 bound planes (reading in kb_oracle.c): [N][H][W + span - 1], entry x + span - 1
    holding the largest max(psi, 0)^2 / phi over the columns [x, x + span) in the image."""
    lib = _load()
    psi = _c(psi, np.float64)
    phi = _c(phi, np.float64)
    N, H, W = psi.shape
    r = np.empty((N, H, W + span - 1), np.float64)
    lib.kbo_snr2_span_max(_ptr(psi), _ptr(phi), N, H, W, int(span), _ptr(r))
    return r


def span_bound(r, W, span, dx_v, dy_v, x0, y0):
    """Upper bound on nu^2 of the trajectories starting in [x0, x0 + span) of row y0 (Psi > 0)."""
    lib = _load()
    r = _c(r, np.float64)
    N, H = r.shape[0], r.shape[1]
    dx_v = _c(dx_v, np.int32)
    dy_v = _c(dy_v, np.int32)
    return lib.kbo_span_bound(_ptr(r), N, H, int(W), int(span), _ptr(dx_v), _ptr(dy_v), int(x0), int(y0))


def search_region(psi, phi, times, dx, dy, k, nu_min=-np.inf, region=None):
    """Top-k records [rows][cols][k] (REC_DTYPE) for start pixels in region=(x_lo, x_hi, y_lo, y_hi)."""
    lib = _load()
    psi = _c(psi, np.float64)
    phi = _c(phi, np.float64)
    times = _c(times, np.float64)
    dx = _c(dx, np.int32)
    dy = _c(dy, np.int32)
    N, H, W = psi.shape
    V = dx.shape[0]
    x_lo, x_hi, y_lo, y_hi = region if region is not None else (0, W, 0, H)
    out = np.empty((y_hi - y_lo, x_hi - x_lo, k), REC_DTYPE)
    lib.kbo_search_region(_ptr(psi), _ptr(phi), _ptr(times), N, H, W, _ptr(dx), _ptr(dy), V, int(k),
                          float(nu_min), x_lo, x_hi, y_lo, y_hi, _ptr(out))
    return out


def search_pixels(psi, phi, times, dx, dy, k, px, py, nu_min=-np.inf):
    """Top-k records [npix][k] for the start pixels (px[i], py[i])."""
    lib = _load()
    psi = _c(psi, np.float64)
    phi = _c(phi, np.float64)
    times = _c(times, np.float64)
    dx = _c(dx, np.int32)
    dy = _c(dy, np.int32)
    px = _c(px, np.int32)
    py = _c(py, np.int32)
    N, H, W = psi.shape
    V = dx.shape[0]
    out = np.empty((px.size, k), REC_DTYPE)
    lib.kbo_search_pixels(_ptr(psi), _ptr(phi), _ptr(times), N, H, W, _ptr(dx), _ptr(dy), V, int(k),
                          float(nu_min), _ptr(px), _ptr(py), px.size, _ptr(out))
    return out


def trajectory_from_images(sci, var, mask, psf, times, dx_v, dy_v, x0, y0, bright_max=None):
    """(Psi, Phi, nobs) of one trajectory computed straight from the raw inputs."""
    lib = _load()
    sci = _c(sci, np.float32)
    var = _c(var, np.float32)
    mask = None if mask is None else _c(mask, np.uint8)
    psf = _c(psf, np.float32)
    times = _c(times, np.float64)
    dx_v = _c(dx_v, np.int32)
    dy_v = _c(dy_v, np.int32)
    N, H, W = sci.shape
    K = psf.shape[-1]
    P = ctypes.c_double()
    F = ctypes.c_double()
    n = ctypes.c_int32()
    lib.kbo_trajectory_from_images(_ptr(sci), _ptr(var), _ptr(mask), _ptr(psf), _ptr(times), N, H, W, K,
                                   _bright(bright_max), _ptr(dx_v), _ptr(dy_v), int(x0), int(y0),
                                   ctypes.byref(P), ctypes.byref(F), ctypes.byref(n))
    return P.value, F.value, n.value


def search_pixels_from_images(sci, var, mask, psf, times, dx, dy, k, px, py, nu_min=-np.inf, bright_max=None):
    """Top-k records [npix][k] at start pixels (px[i], py[i]) computed from the raw images."""
    lib = _load()
    sci = _c(sci, np.float32)
    var = _c(var, np.float32)
    mask = None if mask is None else _c(mask, np.uint8)
    psf = _c(psf, np.float32)
    times = _c(times, np.float64)
    dx = _c(dx, np.int32)
    dy = _c(dy, np.int32)
    px = _c(px, np.int32)
    py = _c(py, np.int32)
    N, H, W = sci.shape
    K = psf.shape[-1]
    V = dx.shape[0]
    out = np.empty((px.size, k), REC_DTYPE)
    lib.kbo_search_pixels_from_images(_ptr(sci), _ptr(var), _ptr(mask), _ptr(psf), _ptr(times), N, H, W, K,
                                      _bright(bright_max), _ptr(dx), _ptr(dy), V, int(k), float(nu_min),
                                      _ptr(px), _ptr(py), px.size, _ptr(out))
    return out
