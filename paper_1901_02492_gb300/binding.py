"""Thin ctypes binding of libkb (include/kb.h): argument marshalling only.

Every step of the search runs in the library's CUDA kernels; this module only
turns torch tensors / numpy arrays into pointers, sizes and a cudaStream_t and
raises KBError on a non-zero status.  There is no CPU fallback: importing it
fails when libkb.so has not been built.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# KB_LIBRARY selects another build of the same library, e.g. libkb_debug.so
LIB_PATH = os.environ.get("KB_LIBRARY") or os.path.join(_HERE, "libkb.so")

KB_OK, KB_EINVAL, KB_ENOMEM, KB_ECUDA, KB_ETIMEOUT, KB_ERANGE = 0, 1, 2, 3, 4, 5
KB_F32, KB_BF16, KB_F16 = 0, 1, 2
KB_RESCORE_FP64 = 1
KB_PRUNE = 2
KB_BATCH_AUTOTUNE = 1
STORAGE = {"f32": KB_F32, "bf16": KB_BF16, "f16": KB_F16}

RESULT_DTYPE = np.dtype([("x0", "<i4"), ("y0", "<i4"), ("vidx", "<i4"), ("nobs", "<i4"),
                         ("vx", "<f4"), ("vy", "<f4"), ("psi", "<f4"), ("phi", "<f4"),
                         ("nu", "<f8"), ("alpha", "<f8")])
assert RESULT_DTYPE.itemsize == 48

# kb_result_compact: start pixel and velocity implied by the position and the caller's grid
COMPACT_DTYPE = np.dtype([("psi", "<f4"), ("phi", "<f4"), ("nu", "<f4"), ("vidx", "<u2"), ("nobs", "u1"),
                          ("reserved", "u1")])
assert COMPACT_DTYPE.itemsize == 16

FILTERED_DTYPE = np.dtype([("x0", "<i4"), ("y0", "<i4"), ("vidx", "<i4"), ("nobs", "<i4"), ("nrejected", "<i4"),
                           ("reserved", "<i4"), ("rejected", "<u4", (4,)), ("psi", "<f8"), ("phi", "<f8"),
                           ("nu", "<f8"), ("alpha", "<f8")])
assert FILTERED_DTYPE.itemsize == 72

MOMENTS_DTYPE = np.dtype([("m00", "<f8"), ("mx", "<f8"), ("my", "<f8"), ("mu20", "<f8"), ("mu02", "<f8"),
                          ("mu11", "<f8"), ("passed", "<i4"), ("reserved", "<i4")])
assert MOMENTS_DTYPE.itemsize == 56
KB_STAMP_MEAN, KB_STAMP_MEDIAN, KB_MAX_STAMP_RADIUS = 0, 1, 15

if not os.path.exists(LIB_PATH):
    raise ImportError("%s is not built (run paper_1901_02492_gb300.build.build() or "
                      "__graft_entry__.build()); there is no fallback path" % LIB_PATH)

_lib = ctypes.CDLL(LIB_PATH)
_P = ctypes.c_void_p
_i32, _f32, _sz = ctypes.c_int, ctypes.c_float, ctypes.c_size_t


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_kb_init = _sig("kb_init", _i32, [ctypes.POINTER(_P), _i32, _sz])
_kb_destroy = _sig("kb_destroy", None, [_P])
_kb_last_error = _sig("kb_last_error", ctypes.c_char_p, [_P])
_kb_hbm_in_use = _sig("kb_hbm_in_use", _sz, [_P])
_kb_debug_build = _sig("kb_debug_build", _i32, [])
_kb_debug_word = _sig("kb_debug_word", _i32, [_P, _P, _i32])
_kb_set_search_variant = _sig("kb_set_search_variant", _i32, [_P, _i32])
_kb_set_search_carveout = _sig("kb_set_search_carveout", _i32, [_P, _i32])
_kb_set_search_swizzle = _sig("kb_set_search_swizzle", _i32, [_P, _i32])
_kb_set_search_order = _sig("kb_set_search_order", _i32, [_P, _i32])
_kb_measure_gather_peak = _sig("kb_measure_gather_peak", _i32, [_P, _i32, _i32, ctypes.POINTER(ctypes.c_double)])
_kb_stack_create = _sig("kb_stack_create", _i32, [_P, _i32, _i32, _i32, _i32, ctypes.POINTER(_P)])
_kb_stack_free = _sig("kb_stack_free", None, [_P])
_kb_make_psi_phi = _sig("kb_make_psi_phi", _i32, [_P, _P, _P, _P, _P, _i32, _f32, _P])
_kb_stack_copy_planes = _sig("kb_stack_copy_planes", _i32, [_P, _i32, _P, _sz, _P])
_kb_stack_scales = _sig("kb_stack_scales", _i32, [_P, _P, _P])
_kb_offsets = _sig("kb_offsets", _i32, [_P, _i32, _P, _P, _i32, _P, _P])
_kb_job_create = _sig("kb_job_create", _i32, [_P, _i32, _i32, _i32, _i32, _i32, _i32, ctypes.POINTER(_P)])
_kb_job_free = _sig("kb_job_free", None, [_P])
_kb_search = _sig("kb_search", _i32, [_P, _P, _P, _P, _P, _i32, _i32, _f32, _i32, _P])
_kb_results = _sig("kb_results", _i32, [_P, _P, _sz, ctypes.POINTER(_sz), _P])
_kb_job_wait = _sig("kb_job_wait", _i32, [_P])
_kb_job_repaired = _sig("kb_job_repaired", _i32, [_P, ctypes.POINTER(_sz)])
_kb_make_psi_phi_static = _sig("kb_make_psi_phi_static", _i32,
                               [_P, _P, _P, _P, _i32, _i32, _i32, _i32, _f32, _P, _P])

_kb_estimate_bytes = _sig("kb_estimate_bytes", _i32, [_i32, _i32, _i32, _i32, _i32, _i32, _i32, _i32,
                                                       ctypes.POINTER(_sz), ctypes.POINTER(_sz)])
_kb_filter_lightcurves = _sig("kb_filter_lightcurves", _i32, [_P, _P, ctypes.c_double, _P, _sz, ctypes.POINTER(_sz), _P])
_kb_stamps = _sig("kb_stamps", _i32, [_P, _P, _P, _i32, _i32, _i32, _P, _P, _P, _i32, _i32, _i32, ctypes.c_double,
                                      _P, _P, _P,
                                      _P])
_kb_results_async = _sig("kb_results_async", _i32, [_P, _P, _sz, ctypes.POINTER(_sz), _P])
_kb_results_compact_async = _sig("kb_results_compact_async", _i32, [_P, _P, _sz, ctypes.POINTER(_sz), _P])
_kb_cluster = _sig("kb_cluster", _i32, [_P, _P, _sz, _P, _P, _P, _P, ctypes.POINTER(_sz), _P])
_kb_batch_create = _sig("kb_batch_create", _i32, [_P, _i32, _P, _i32, ctypes.POINTER(_P)])
_kb_batch_run = _sig("kb_batch_run", _i32, [_P, _P])
_kb_batch_groups = _sig("kb_batch_groups", _i32, [_P, _P, _i32, ctypes.POINTER(_i32)])
_kb_batch_free = _sig("kb_batch_free", None, [_P])

EXPORTED = ["kb_init", "kb_destroy", "kb_last_error", "kb_hbm_in_use", "kb_debug_build", "kb_debug_word",
            "kb_set_search_variant",
            "kb_set_search_carveout", "kb_set_search_swizzle", "kb_set_search_order", "kb_measure_gather_peak", "kb_stack_create", "kb_stack_free",
            "kb_make_psi_phi", "kb_stack_copy_planes", "kb_stack_scales", "kb_offsets", "kb_job_create",
            "kb_job_free", "kb_search", "kb_job_wait", "kb_job_repaired", "kb_results", "kb_make_psi_phi_static",
            "kb_batch_create", "kb_batch_run", "kb_batch_groups", "kb_batch_free", "kb_estimate_bytes",
            "kb_filter_lightcurves", "kb_stamps", "kb_cluster", "kb_results_async", "kb_results_compact_async"]


class ClusterParams(ctypes.Structure):
    """kb_cluster_params: weights of the start pixel and velocity coordinates, eps, min_samples."""
    _fields_ = [("w_pos", ctypes.c_double), ("w_vel", ctypes.c_double), ("eps", ctypes.c_double),
                ("min_samples", _i32), ("reserved", _i32)]


class MomentCuts(ctypes.Structure):
    """kb_moment_cuts: a stamp passes when m00 > 0, |mx|, |my| <= max_offset,
    min_var <= mu20, mu02 <= max_var and |mu11| <= max_mu11."""
    _fields_ = [("max_offset", ctypes.c_double), ("min_var", ctypes.c_double), ("max_var", ctypes.c_double),
                ("max_mu11", ctypes.c_double)]


class KBError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("kb status %d: %s" % (code, msg))
        self.code = code


def _ptr(x):
    """Data pointer of a torch tensor or numpy array (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Context:
    """kb_ctx: one CUDA device and an HBM budget (0 = none)."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        h = _P()
        rc = _kb_init(ctypes.byref(h), int(device), int(hbm_budget))
        if rc != KB_OK:
            raise KBError(rc, "kb_init(device=%d) failed" % device)
        self.h = h
        self.device = device

    def check(self, rc):
        if rc != KB_OK:
            raise KBError(rc, _kb_last_error(self.h).decode())

    @property
    def last_error(self) -> str:
        return _kb_last_error(self.h).decode()

    def set_search_variant(self, variant: int):
        self.check(_kb_set_search_variant(self.h, int(variant)))

    def set_search_carveout(self, percent: int):
        self.check(_kb_set_search_carveout(self.h, int(percent)))

    def set_search_swizzle(self, cols: int):
        """Search tile order: super-columns of `cols` tiles (-1 automatic, 0 row by row)."""
        self.check(_kb_set_search_swizzle(self.h, int(cols)))

    def set_search_order(self, order: int):
        """Velocity order: 0 by latest (dy, dx), 1 Hilbert over latest offsets, 2 the caller's, -1 automatic."""
        self.check(_kb_set_search_order(self.h, int(order)))

    def measure_gather_peak(self, warp_bytes: int = 512, align_bytes: int = 8) -> float:
        """L2-to-SM GB/s of the search's access form on this device (roofline denominator): warps
        reading warp_bytes contiguous bytes at scattered multiples of align_bytes."""
        v = ctypes.c_double()
        self.check(_kb_measure_gather_peak(self.h, int(warp_bytes), int(align_bytes), ctypes.byref(v)))
        return v.value

    @property
    def hbm_in_use(self) -> int:
        return int(_kb_hbm_in_use(self.h))

    def debug_word(self, reset: bool = True) -> int:
        """KB_DEBUG builds: the first out-of-bounds access the search kernels met,
        (site << 56) | offset, 0 if none (kb_debug_word)."""
        w = ctypes.c_ulonglong(0)
        self.check(_kb_debug_word(self.h, ctypes.byref(w), 1 if reset else 0))
        return int(w.value)

    def cluster(self, cand, w_pos, w_vel, eps, min_samples, core=False, stream=None):
        """Sec. 3.3 DBSCAN de-duplication of device kb_result records `cand` (a CUDA tensor
        holding RESULT_DTYPE records).  Returns (label int32, keep bool, core bool or None) as
        device tensors and the number of groups."""
        import torch
        nbytes = cand.numel() * cand.element_size()
        if nbytes % RESULT_DTYPE.itemsize or not cand.is_contiguous():
            raise ValueError("cand must be a contiguous tensor of kb_result records")
        n = nbytes // RESULT_DTYPE.itemsize
        dev = cand.device
        label = torch.empty(n, dtype=torch.int32, device=dev)
        keep = torch.empty(n, dtype=torch.uint8, device=dev)
        cor = torch.empty(n, dtype=torch.uint8, device=dev) if core else None
        p = ClusterParams(float(w_pos), float(w_vel), float(eps), int(min_samples), 0)
        groups = _sz()
        self.check(_kb_cluster(self.h, _ptr(cand), n, ctypes.byref(p), _ptr(label), _ptr(keep), _ptr(cor),
                               ctypes.byref(groups), _stream(stream)))
        return label, keep.bool(), None if cor is None else cor.bool(), int(groups.value)

    def close(self):
        if self.h:
            _kb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stack:
    """kb_stack: device-resident psi/phi planes of an N x H x W stack."""

    def __init__(self, ctx: Context, N: int, H: int, W: int, storage="f32"):
        self.ctx = ctx
        self.N, self.H, self.W = N, H, W
        self.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        h = _P()
        ctx.check(_kb_stack_create(ctx.h, N, H, W, self.storage, ctypes.byref(h)))
        self.h = h

    def make_psi_phi(self, sci, var, mask, psf, bright_max=math.inf, stream=None):
        """sci/var: CUDA float32 [N][H][W]; mask: CUDA uint8 or None; psf: host float32 [N][K][K]."""
        psf = np.ascontiguousarray(psf, dtype=np.float32)
        K = psf.shape[-1]
        self.ctx.check(_kb_make_psi_phi(self.h, _ptr(sci), _ptr(var), _ptr(mask), psf.ctypes.data, K,
                                        float(bright_max), _stream(stream)))

    def copy_planes(self, which: int, dst, stream=None):
        nbytes = dst.numel() * dst.element_size() if hasattr(dst, "numel") else dst.nbytes
        self.ctx.check(_kb_stack_copy_planes(self.h, which, _ptr(dst), nbytes, _stream(stream)))

    def scales(self):
        sp = np.empty(self.N, np.float32)
        sf = np.empty(self.N, np.float32)
        self.ctx.check(_kb_stack_scales(self.h, sp.ctypes.data, sf.ctypes.data))
        return sp, sf

    def free(self):
        if self.h:
            _kb_stack_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def _check_device_tensor(name, t, dtype, numel, device):
    """The C entry point gets raw pointers and no buffer sizes, so the wrapper checks each
    buffer before the call: a CUDA tensor on the given device, contiguous, of the given
    dtype and element count."""
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.device != device:
        raise ValueError("%s is on %s, not on %s" % (name, t.device, device))
    if t.numel() != numel:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), numel))


def make_psi_phi_static(sci, var, mask, psf, out, bright_max=math.inf, stream=None):
    """psi/phi planes into the caller's device buffer `out` (float32 [N][H][W][2]) without any
    allocation: the PSF taps go to the library's static device scratch (see include/kb.h).
    sci, var: float32 CUDA tensors [N][H][W]; mask: uint8 [N][H][W] or None; psf: host
    [N][K][K]; all on the current CUDA device.  Nothing is launched unless every buffer
    matches (N, H, W)."""
    import torch
    psf = np.ascontiguousarray(psf, dtype=np.float32)
    if psf.ndim != 3 or psf.shape[1] != psf.shape[2]:
        raise ValueError("psf must be [N][K][K], got shape %s" % (psf.shape,))
    if not isinstance(sci, torch.Tensor) or sci.dim() != 3:
        raise ValueError("sci must be a [N][H][W] tensor")
    N, K = psf.shape[0], psf.shape[-1]
    H, W = sci.shape[-2], sci.shape[-1]
    if sci.shape[0] != N:
        raise ValueError("sci has %d epochs, the psf %d" % (sci.shape[0], N))
    for name, t in (("sci", sci), ("var", var), ("mask", mask), ("out", out)):
        if t is not None and not (isinstance(t, torch.Tensor) and t.is_cuda):
            raise ValueError("%s must be a CUDA tensor" % name)
    dev = torch.device("cuda", torch.cuda.current_device())
    _check_device_tensor("sci", sci, torch.float32, N * H * W, dev)
    _check_device_tensor("var", var, torch.float32, N * H * W, dev)
    if mask is not None:
        _check_device_tensor("mask", mask, torch.uint8, N * H * W, dev)
    _check_device_tensor("out", out, torch.float32, 2 * N * H * W, dev)
    rc = _kb_make_psi_phi_static(_ptr(sci), _ptr(var), _ptr(mask), psf.ctypes.data, N, H, W, K,
                                 float(bright_max), _ptr(out), _stream(stream))
    if rc != KB_OK:
        raise KBError(rc, "kb_make_psi_phi_static failed")


def debug_build() -> bool:
    """Whether the loaded library is a KB_DEBUG build (kb_debug_build)."""
    return bool(_kb_debug_build())


def estimate_bytes(N, H, W, storage, K, V, topk, flags=0):
    """(stack bytes, job bytes) that kb_stack_create + kb_make_psi_phi and kb_job_create will hold."""
    st = STORAGE[storage] if isinstance(storage, str) else int(storage)
    a, b = _sz(), _sz()
    rc = _kb_estimate_bytes(int(N), int(H), int(W), st, int(K), int(V), int(topk), int(flags), ctypes.byref(a),
                            ctypes.byref(b))
    if rc != KB_OK:
        raise KBError(rc, "kb_estimate_bytes rejected the shape")
    return int(a.value), int(b.value)


def offsets(times, vx, vy):
    """The library's fixed-point trajectory offsets: dx, dy int32 [V][N]."""
    times, vx, vy = _f64(times), _f64(vx), _f64(vy)
    N, V = times.size, vx.size
    dx = np.empty((V, N), np.int32)
    dy = np.empty((V, N), np.int32)
    rc = _kb_offsets(times.ctypes.data, N, vx.ctypes.data, vy.ctypes.data, V, dx.ctypes.data, dy.ctypes.data)
    if rc != KB_OK:
        raise KBError(rc, "kb_offsets rejected the times or velocities")
    return dx, dy


class Job:
    """kb_job: device results of searches over H x W start pixels."""

    def __init__(self, ctx: Context, H: int, W: int, N: int, V: int, topk: int, flags: int = 0):
        self.ctx = ctx
        self.H, self.W, self.topk = H, W, topk
        h = _P()
        ctx.check(_kb_job_create(ctx.h, H, W, N, V, topk, flags, ctypes.byref(h)))
        self.h = h
        self.k = None

    def search(self, stack: Stack, times, vx, vy, topk=None, nu_min=-math.inf, flags=0, stream=None):
        times, vx, vy = _f64(times), _f64(vx), _f64(vy)
        topk = self.topk if topk is None else topk
        self.ctx.check(_kb_search(self.h, stack.h, times.ctypes.data, vx.ctypes.data, vy.ctypes.data, vx.size,
                                  int(topk), float(nu_min), int(flags), _stream(stream)))
        self.k = topk

    def wait(self):
        """Wait for the last search; raises KBError(KB_ETIMEOUT) if a device wait gave up."""
        self.ctx.check(_kb_job_wait(self.h))

    def repaired(self) -> int:
        """Pixels re-searched in FP64 because the rescoring certificate could not clear them."""
        n = _sz()
        self.ctx.check(_kb_job_repaired(self.h, ctypes.byref(n)))
        return int(n.value)

    def results(self, out=None, stream=None):
        """Records [H][W][k] of RESULT_DTYPE.  out: None (new numpy array), a numpy array of
        RESULT_DTYPE, or a CUDA uint8 tensor of >= H*W*k*48 bytes (device output)."""
        n = self.H * self.W * self.k
        if out is None:
            out = np.empty(n, RESULT_DTYPE)
        if hasattr(out, "numel"):
            cap = out.numel() * out.element_size() // RESULT_DTYPE.itemsize
        else:
            cap = out.nbytes // RESULT_DTYPE.itemsize
        written = _sz()
        self.ctx.check(_kb_results(self.h, _ptr(out), cap, ctypes.byref(written), _stream(stream)))
        if isinstance(out, np.ndarray):
            return out.reshape(self.H, self.W, self.k)
        return out

    def results_async(self, out, stream=None):
        """Enqueue the records [H][W][k] into `out` (a CUDA uint8 tensor, or page-locked host memory:
        a pinned torch tensor or a numpy view of one) on `stream` without waiting; `out` is
        complete once the stream reaches this point."""
        cap = (out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes) // RESULT_DTYPE.itemsize
        written = _sz()
        self.ctx.check(_kb_results_async(self.h, _ptr(out), cap, ctypes.byref(written), _stream(stream)))
        return out

    def results_compact_async(self, out, stream=None):
        """Enqueue the compact records [H][W][k] (COMPACT_DTYPE, 16 bytes each) into `out` (a CUDA
        uint8 tensor or page-locked host memory) on `stream` without waiting."""
        cap = (out.numel() * out.element_size() if hasattr(out, "numel") else out.nbytes) // COMPACT_DTYPE.itemsize
        written = _sz()
        self.ctx.check(_kb_results_compact_async(self.h, _ptr(out), cap, ctypes.byref(written), _stream(stream)))
        return out

    def filter_lightcurves(self, stack: Stack, nsigma=5.0, out=None, stream=None):
        """Sec. 3.3 outlier filter of the kept trajectories: FILTERED_DTYPE records [H][W][k].
        out: None (returned as numpy, through a temporary device buffer) or a CUDA uint8 tensor."""
        import torch
        n = self.H * self.W * (self.k or self.topk)
        dev = out
        if dev is None:
            dev = torch.empty(n * FILTERED_DTYPE.itemsize, dtype=torch.uint8, device="cuda:%d" % self.ctx.device)
        cap = dev.numel() * dev.element_size() // FILTERED_DTYPE.itemsize
        written = _sz()
        self.ctx.check(_kb_filter_lightcurves(self.h, stack.h, float(nsigma), _ptr(dev), cap, ctypes.byref(written),
                                              _stream(stream)))
        if out is None:
            return dev.cpu().numpy().view(FILTERED_DTYPE).reshape(self.H, self.W, self.k or self.topk)
        return out

    def stamps(self, sci, mask, x0, y0, vidx, radius, median=False, cuts=None, moments=True, stream=None,
               aperture=0.0):
        """Sec. 3.3 coadded stamps of candidates (x0, y0, vidx) of the last search from the device
        science images sci [N][H][W] (float32) and mask (uint8 or None).  Returns the device
        stamps [n][2r+1][2r+1] (float32) and, with moments, a MOMENTS_DTYPE numpy array [n] of the
        moments over the central aperture (radius `aperture` px; <= 0: the whole stamp).
        cuts: None or a MomentCuts (or a dict of its fields)."""
        import torch
        x0 = np.ascontiguousarray(x0, np.int32)
        y0 = np.ascontiguousarray(y0, np.int32)
        vidx = np.ascontiguousarray(vidx, np.int32)
        n = x0.size
        if y0.size != n or vidx.size != n:
            raise ValueError("x0, y0 and vidx differ in length")
        N, H, W = sci.shape
        if sci.dtype != torch.float32 or not sci.is_contiguous():
            raise ValueError("sci must be a contiguous float32 [N][H][W] tensor")
        if mask is not None and (mask.dtype != torch.uint8 or not mask.is_contiguous() or mask.shape != sci.shape):
            raise ValueError("mask must be a contiguous uint8 tensor of the images' shape")
        S = 2 * int(radius) + 1
        dev = sci.device
        st = torch.empty((n, S, S), dtype=torch.float32, device=dev)
        mo = torch.empty(n * MOMENTS_DTYPE.itemsize, dtype=torch.uint8, device=dev) if moments else None
        if isinstance(cuts, dict):
            cuts = MomentCuts(**cuts)
        self.ctx.check(_kb_stamps(self.h, _ptr(sci), _ptr(mask), N, H, W, _ptr(x0), _ptr(y0), _ptr(vidx), n,
                                  int(radius), KB_STAMP_MEDIAN if median else KB_STAMP_MEAN, float(aperture),
                                  None if cuts is None else ctypes.byref(cuts), _ptr(st), _ptr(mo), _stream(stream)))
        if mo is None:
            return st, None
        return st, mo.cpu().numpy().view(MOMENTS_DTYPE)

    def free(self):
        if self.h:
            _kb_job_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass



class _BatchItem(ctypes.Structure):
    _fields_ = [("job", _P), ("stack", _P), ("times", _P), ("vx", _P), ("vy", _P), ("V", _i32),
                ("topk", _i32), ("nu_min", _f32), ("flags", _i32)]


class BatchGroup(ctypes.Structure):
    """kb_batch_group: the plan of one persistent launch of a batch."""
    _fields_ = [("storage", _i32), ("index_bits", _i32), ("variant", _i32), ("kmax", _i32),
                ("n_items", ctypes.c_longlong), ("evals", ctypes.c_double), ("tuned_ms", _f32 * 5),
                ("schedule", _i32), ("tuned_ms_launch", _f32 * 5)]


class Batch:
    """kb_batch: many searches (job, stack, times, vx, vy, topk, nu_min, flags) as one graph-captured,
    persistent launch per storage group.  `searches` is a list of dicts with those keys."""

    def __init__(self, ctx: Context, searches, autotune=True):
        self.ctx = ctx
        self._keep = []
        arr = (_BatchItem * len(searches))()
        for i, d in enumerate(searches):
            times, vx, vy = _f64(d["times"]), _f64(d["vx"]), _f64(d["vy"])
            self._keep += [times, vx, vy]
            job = d["job"]
            topk = int(d.get("topk", job.topk))
            arr[i] = _BatchItem(job.h, d["stack"].h, times.ctypes.data, vx.ctypes.data, vy.ctypes.data, vx.size,
                                topk, float(d.get("nu_min", -math.inf)), int(d.get("flags", 0)))
            job.k = topk
        self.jobs = [d["job"] for d in searches]
        h = _P()
        ctx.check(_kb_batch_create(ctx.h, len(searches), ctypes.cast(arr, _P),
                                   KB_BATCH_AUTOTUNE if autotune else 0, ctypes.byref(h)))
        self.h = h
        self._keep = None

    def run(self, stream=None):
        self.ctx.check(_kb_batch_run(self.h, _stream(stream)))

    def groups(self):
        n = _i32()
        self.ctx.check(_kb_batch_groups(self.h, None, 0, ctypes.byref(n)))
        out = (BatchGroup * n.value)()
        self.ctx.check(_kb_batch_groups(self.h, ctypes.cast(out, _P), n.value, ctypes.byref(n)))
        return list(out)

    def free(self):
        if self.h:
            _kb_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
