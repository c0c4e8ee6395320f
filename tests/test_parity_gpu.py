"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Small cases are compared element by element (psi/phi planes, every top-k slot);
they span several kernel tiles (psi/phi 64x32, search 128x8 start pixels) and
ragged tails.  The full DECam-shaped 12 x 4096 x 4096 search is checked on
sampled start pixels that the oracle recomputes from the raw images.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from _compare import NU_RTOL, check_topk, nu_tol, oracle_nu_table

pytestmark = pytest.mark.gpu
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def ctx(kb):
    c = kb.Context(0)
    yield c
    c.close()


def to_dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def gpu_planes(kb, ctx, st, storage="f32", bright=math.inf, mask=True):
    N, H, W = st.sci.shape
    s = kb.Stack(ctx, N, H, W, storage)
    s.make_psi_phi(to_dev(st.sci), to_dev(st.var), to_dev(st.mask) if mask else None, st.psf, bright)
    return s


def gpu_search(kb, ctx, st, storage="f32", k=None, nu_min=-math.inf, flags=0, times=None, vx=None, vy=None,
               bright=math.inf):
    """Search through the C ABI and return the kb_result records [H][W][k]."""
    N, H, W = st.sci.shape
    k = st.k if k is None else k
    times = st.times if times is None else times
    vx = st.vx if vx is None else vx
    vy = st.vy if vy is None else vy
    s = gpu_planes(kb, ctx, st, storage, bright)
    job = kb.Job(ctx, H, W, N, len(vx), k, flags)
    job.search(s, times, vx, vy, k, nu_min, flags)
    res = job.results()
    torch.cuda.synchronize()
    job.free()
    s.free()
    return res


def oracle_search(st, k=None, nu_min=-np.inf, times=None, vx=None, vy=None, bright=None):
    k = st.k if k is None else k
    times = st.times if times is None else times
    vx = st.vx if vx is None else vx
    vy = st.vy if vy is None else vy
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf, bright)
    dx, dy = oracle.offsets(times, vx, vy)
    ref = oracle.search_region(psi, phi, times, dx, dy, k, nu_min)
    table = oracle_nu_table(psi, phi, times, dx, dy)
    return ref, (lambda p, v: table[p, v])


# ------------------------------------------------------------------ stage (a)

def _asym(K, seed):
    rng = np.random.default_rng(seed)
    p = rng.uniform(0.1, 1.0, (K, K)).astype(np.float32)
    return (p / p.sum()).astype(np.float32)


@pytest.mark.parametrize("K,sep,mask,bright", [(7, True, False, math.inf), (17, True, True, math.inf),
                                               (5, False, True, 40.0), (1, True, False, math.inf),
                                               (31, True, False, math.inf)])
def test_psi_phi_planes_f32(kb, ctx, K, sep, mask, bright):
    st = synth.small_stack(100 + K, 3, 77, 150, K=K, sigma=max(K / 6.0, 0.5), var_lo=50, var_hi=150,
                           nan_frac=0.01, mask_frac=0.02 if mask else 0.0, flux=400.0)
    if not sep:
        st.psf = np.stack([_asym(K, e) for e in range(st.psf.shape[0])])
    s = gpu_planes(kb, ctx, st, bright=bright)
    N, H, W = st.sci.shape
    out = torch.empty((N, H, W, 2), dtype=torch.float32, device=DEV)
    s.copy_planes(0, out)
    g = out.cpu().numpy()
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf, None if math.isinf(bright) else bright)
    scale = np.abs(psi) + np.sqrt(phi)
    assert np.all(np.abs(g[..., 0] - psi) <= 1e-5 * scale + 1e-30)
    assert np.all(np.abs(g[..., 1] - phi) <= 1e-5 * phi + 1e-30)
    assert np.array_equal(g[..., 1] == 0, phi == 0)
    s.free()


@pytest.mark.parametrize("K,mask,H,W", [(3, False, 77, 152), (7, True, 77, 152), (17, True, 77, 152),
                                         (15, False, 45, 200), (17, False, 1100, 68), (21, False, 45, 200),
                                         (17, True, 70, 1000), (5, False, 1030, 508)])
def test_psi_phi_stream_kernel(kb, ctx, K, mask, H, W):
    """Separable PSFs (K <= 21) on widths divisible by 4 take the streaming kernel (column
    strips walked down segments of up to 512 rows, in batches of 32 rows; the last two cases
    span many strips, and the second also several segments); other widths the tile kernel.
    Planes against the oracle, and bit for bit against the tile kernel: the same stack with
    one more column, of NaN variance (weight 0, like the outside of the image), goes to the
    tile kernel."""
    st = synth.small_stack(300 + K, 3, H, W, K=K, sigma=max(K / 6.0, 0.5), var_lo=50, var_hi=150,
                           nan_frac=0.01, mask_frac=0.02 if mask else 0.0, flux=400.0)
    N = st.sci.shape[0]
    planes = []
    for extra in (0, 1):
        sci = np.concatenate([st.sci, np.zeros((N, H, extra), np.float32)], axis=2)
        var = np.concatenate([st.var, np.full((N, H, extra), np.nan, np.float32)], axis=2)
        msk = None if st.mask is None else np.concatenate([st.mask, np.zeros((N, H, extra), np.uint8)], axis=2)
        s = kb.Stack(ctx, N, H, W + extra, "f32")
        s.make_psi_phi(to_dev(sci), to_dev(var), to_dev(msk) if msk is not None else None, st.psf)
        out = torch.empty((N, H, W + extra, 2), dtype=torch.float32, device=DEV)
        s.copy_planes(0, out)
        planes.append(out.cpu().numpy()[:, :, :W])
        s.free()
    assert planes[0].tobytes() == planes[1].tobytes()
    psi, phi = oracle.psi_phi(st.sci, st.var, st.mask, st.psf)
    g = planes[0]
    assert np.all(np.abs(g[..., 0] - psi) <= 1e-5 * (np.abs(psi) + np.sqrt(phi)) + 1e-30)
    assert np.all(np.abs(g[..., 1] - phi) <= 1e-5 * phi + 1e-30)
    assert np.array_equal(g[..., 1] == 0, phi == 0)


# ------------------------------------------------------------------ stage (b), FP32

@pytest.mark.parametrize("k", [1, 4, 8, 16])
def test_search_f32_small(kb, ctx, k):
    st = synth.small_stack(7, 5, 70, 150, K=7, nan_frac=0.01, n_angles=8, n_speeds=8, s_hi=12.0,
                           n_sources=3, flux=40.0)
    res = gpu_search(kb, ctx, st, k=k)
    ref, nu_of = oracle_search(st, k=k)
    check_topk(res, ref, nu_of)


def test_search_tiny_workload(kb, ctx):
    """The 5 x 64 x 64 workload: full comparison of every slot."""
    st = synth.tiny()
    res = gpu_search(kb, ctx, st)
    ref, nu_of = oracle_search(st)
    check_topk(res, ref, nu_of)
    assert np.array_equal(res["x0"][5, 7], np.full(st.k, 7)) and np.array_equal(res["y0"][5, 7], np.full(st.k, 5))


EDGE_CASES = {
    "one_epoch": dict(N=1, H=20, W=33),
    "one_row": dict(N=4, H=1, W=300),
    "one_column": dict(N=4, H=50, W=1),
    "ragged": dict(N=6, H=13, W=37),
    "wide_ragged": dict(N=3, H=9, W=261),
    "same_time": dict(N=3, H=16, W=40, times=[1.0, 1.0, 1.0]),
    "unordered_times": dict(N=4, H=24, W=70, times=[2.0, 0.5, 1.25, 0.5]),
    "fast_off_image": dict(N=4, H=30, W=40, s_lo=30.0, s_hi=60.0),
}


@pytest.mark.parametrize("name", sorted(EDGE_CASES))
def test_search_edge_cases(kb, ctx, name):
    c = dict(EDGE_CASES[name])
    times = c.pop("times", None)
    st = synth.small_stack(11, c.pop("N"), c.pop("H"), c.pop("W"), K=5, nan_frac=0.02, n_angles=6,
                           n_speeds=5, times=times, **c)
    res = gpu_search(kb, ctx, st, k=3)
    ref, nu_of = oracle_search(st, k=3)
    check_topk(res, ref, nu_of)


def test_search_threshold_and_masked_epoch(kb, ctx):
    st = synth.small_stack(12, 4, 40, 90, K=5, mask_frac=0.05, n_sources=2, flux=30.0)
    st.var[1, :, :30] = -1.0          # a fully masked band in one epoch
    res = gpu_search(kb, ctx, st, k=5, nu_min=1.0)
    ref, nu_of = oracle_search(st, k=5, nu_min=1.0)
    check_topk(res, ref, nu_of)
    assert np.all(res["nu"][res["vidx"] >= 0] >= 1.0)


def test_search_single_velocity_and_duplicates(kb, ctx):
    st = synth.small_stack(13, 5, 33, 65, K=5)
    vx = np.array([3.0, 3.0, 3.01, -2.0])
    vy = np.array([1.0, 1.0, 1.0, 0.5])
    res = gpu_search(kb, ctx, st, k=4, vx=vx, vy=vy)
    ref, nu_of = oracle_search(st, k=4, vx=vx, vy=vy)
    check_topk(res, ref, nu_of, max_mismatch_frac=0.0)
    one = gpu_search(kb, ctx, st, k=2, vx=vx[:1], vy=vy[:1])
    ref1, nu_of1 = oracle_search(st, k=2, vx=vx[:1], vy=vy[:1])
    check_topk(one, ref1, nu_of1)


def test_bright_pixel_limit(kb, ctx):
    st = synth.small_stack(14, 3, 40, 64, K=5, var_lo=100, var_hi=100, n_sources=3, flux=3000.0)
    res = gpu_search(kb, ctx, st, k=3, bright=120.0)
    ref, nu_of = oracle_search(st, k=3, bright=120.0)
    check_topk(res, ref, nu_of)


def test_results_to_device_buffer(kb, ctx):
    st = synth.small_stack(15, 4, 30, 50, K=5)
    N, H, W = st.sci.shape
    s = gpu_planes(kb, ctx, st)
    job = kb.Job(ctx, H, W, N, st.vx.size, 4)
    job.search(s, st.times, st.vx, st.vy, 4)
    host = job.results()
    dev = torch.empty(H * W * 4 * kb.RESULT_DTYPE.itemsize, dtype=torch.uint8, device=DEV)
    job.results(dev)
    torch.cuda.synchronize()
    devh = dev.cpu().numpy().view(kb.RESULT_DTYPE).reshape(H, W, 4)
    assert np.array_equal(host, devh)
    # page-locked host memory is written by the GPU directly: the same records
    pinned = torch.zeros(H * W * 4 * kb.RESULT_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    pin_np = pinned.numpy().view(kb.RESULT_DTYPE)
    job.results(pin_np)
    assert np.array_equal(host.ravel(), pin_np)
    # re-running the same job with a different k and grid reuses its buffers
    job.search(s, st.times, st.vx[:10], st.vy[:10], 2)
    again = job.results()
    ref, nu_of = oracle_search(st, k=2, vx=st.vx[:10], vy=st.vy[:10])
    check_topk(again, ref, nu_of)
    job.free()
    s.free()


def test_api_rejects_bad_arguments(kb, ctx):
    st = synth.small_stack(16, 2, 8, 8, K=3)
    s = kb.Stack(ctx, 2, 8, 8)
    with pytest.raises(kb.KBError) as e:   # K even
        s.make_psi_phi(to_dev(st.sci), to_dev(st.var), None, np.ones((2, 4, 4), np.float32))
    assert e.value.code == kb.KB_EINVAL
    with pytest.raises(kb.KBError) as e:   # host pointers for the images
        s.make_psi_phi(st.sci, st.var, None, st.psf)
    assert e.value.code == kb.KB_EINVAL
    job = kb.Job(ctx, 8, 8, 2, 4, 2)
    with pytest.raises(kb.KBError):        # search before psi/phi exist
        job.search(s, st.times, st.vx[:4], st.vy[:4])
    s.make_psi_phi(to_dev(st.sci), to_dev(st.var), None, st.psf)
    with pytest.raises(kb.KBError):        # more velocities than the job holds
        job.search(s, st.times, st.vx[:5], st.vy[:5])
    with pytest.raises(kb.KBError):        # k above the job's k
        job.search(s, st.times, st.vx[:4], st.vy[:4], topk=3)
    with pytest.raises(kb.KBError) as e:   # velocity outside the fixed-point range
        job.search(s, st.times, np.array([5000.0]), np.array([0.0]))
    assert e.value.code == kb.KB_EINVAL
    with pytest.raises(kb.KBError) as e:
        kb.Job(ctx, 8, 8, 2, 4, 17)
    job.free()
    s.free()


def test_hbm_budget(kb):
    c = kb.Context(0, hbm_budget=1 << 20)
    with pytest.raises(kb.KBError) as e:
        kb.Stack(c, 4, 512, 512)
    assert e.value.code == kb.KB_ENOMEM
    assert c.hbm_in_use == 0
    s = kb.Stack(c, 1, 64, 64)
    assert 0 < c.hbm_in_use <= 1 << 20
    s.free()
    assert c.hbm_in_use == 0
    c.close()


# ------------------------------------------------------------------ full DECam-shaped size

@pytest.fixture(scope="module")
def decam_stack():
    return synth.decam()


def test_decam_full_size_sampled(kb, ctx, decam_stack):
    """12 x 4096 x 4096, 1024 velocities, k = 8 (the benchmark's launch configuration):
    sampled start pixels (corners, edges, injected sources, random) against the oracle."""
    st = decam_stack
    N, H, W = st.sci.shape
    res = gpu_search(kb, ctx, st)
    rng = np.random.default_rng(99)
    px = [0, W - 1, 0, W - 1, W // 2, 1, W - 2] + list(rng.integers(0, W, 90))
    py = [0, 0, H - 1, H - 1, H // 2, H - 2, 1] + list(rng.integers(0, H, 90))
    for s in st.sources[:20]:
        px.append(min(max(int(round(s["x0"])), 0), W - 1))
        py.append(min(max(int(round(s["y0"])), 0), H - 1))
    px, py = np.array(px), np.array(py)
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    ref = oracle.search_pixels_from_images(st.sci, st.var, None, st.psf, st.times, dx, dy, st.k, px, py)
    g = res[py, px]

    def nu_of(p, v):
        P, F, _ = oracle.trajectory_from_images(st.sci, st.var, None, st.psf, st.times, dx[v], dy[v], px[p], py[p])
        return P / math.sqrt(F) if F > 0 else -math.inf
    check_topk(g, ref, nu_of)
    assert np.all(g["x0"] == px[:, None]) and np.all(g["y0"] == py[:, None])


@pytest.mark.parametrize("variant", range(0, 9))
@pytest.mark.parametrize("storage", ["f32", "bf16", "f16"])
def test_every_kernel_variant(kb, ctx, variant, storage):
    """Every search kernel (register gather 0-4, TMA pipeline 5-8) in every shape gives the oracle's
    results: ragged tile edges, masked pixels, trajectories leaving the image, odd and even shifts
    of the 16-bit pixel pairs."""
    st = synth.small_stack(40 + variant, 6, 45, 203, K=5, nan_frac=0.01, mask_frac=0.01, n_angles=6,
                           n_speeds=6, s_lo=5.0, s_hi=40.0, n_sources=2, flux=60.0)
    ctx.set_search_variant(variant)
    try:
        flags = kb.KB_RESCORE_FP64 if storage != "f32" else 0
        res = gpu_search(kb, ctx, st, storage, k=5, flags=flags)
    finally:
        ctx.set_search_variant(0)
    ref, nu_of = oracle_search(st, k=5)
    check_topk(res, ref, nu_of)


def test_results_async_overlaps_and_orders_reads(kb, ctx):
    """kb_results_async into pinned host memory on a second stream equals kb_results; a search
    enqueued right after the read (same job, other velocities) waits for the read, so the
    buffer holds the first search's records; pageable host memory is refused."""
    st = synth.small_stack(91, 6, 90, 140, K=5, nan_frac=0.01, n_angles=8, n_speeds=8, s_hi=12.0, n_sources=3,
                           flux=40.0)
    N, H, W = st.sci.shape
    s = gpu_planes(kb, ctx, st)
    jobs = [kb.Job(ctx, H, W, N, st.vx.size, st.k, 0) for _ in range(2)]
    vx2, vy2 = st.vx[::-1].copy() * 0.5, st.vy[::-1].copy() * 0.5
    n = H * W * st.k * kb.RESULT_DTYPE.itemsize
    pinned = [torch.empty(n, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    s_out = torch.cuda.Stream()
    ref1 = None
    for j in jobs:
        j.search(s, st.times, st.vx, st.vy, st.k, -math.inf, 0)
        ref1 = j.results()
    torch.cuda.synchronize()
    for b, j in enumerate(jobs):
        j.search(s, st.times, st.vx, st.vy, st.k, -math.inf, 0)
        j.results_async(pinned[b], stream=s_out)
        j.search(s, st.times, vx2, vy2, st.k, -math.inf, 0)     # must not overtake the read
    torch.cuda.synchronize()
    for b, j in enumerate(jobs):
        assert pinned[b].numpy().tobytes() == ref1.tobytes()
        ref2 = j.results()
        assert ref2.tobytes() != ref1.tobytes()
        dev = torch.empty(n, dtype=torch.uint8, device=DEV)
        j.results_async(dev)
        torch.cuda.synchronize()
        assert dev.cpu().numpy().tobytes() == ref2.tobytes()
    with pytest.raises(kb.KBError):
        jobs[0].results_async(np.empty(H * W * st.k, kb.RESULT_DTYPE))
    for j in jobs:
        j.free()
    s.free()


def _compact_from_full(kb, full):
    """The compact records a kb_result array implies (FP32 rounding of the FP64 fields)."""
    f = full.reshape(-1)
    c = np.zeros(f.size, kb.COMPACT_DTYPE)
    empty = f["vidx"] < 0
    c["psi"] = np.where(empty, 0.0, f["psi"])
    c["phi"] = np.where(empty, 0.0, f["phi"])
    c["nu"] = np.where(empty, -np.inf, f["nu"].astype(np.float32))
    c["vidx"] = np.where(empty, 0xFFFF, f["vidx"]).astype(np.uint16)
    c["nobs"] = np.where(empty, 0, f["nobs"]).astype(np.uint8)
    return c


@pytest.mark.parametrize("storage,flags", [("f32", 0), ("bf16", 1), ("f16", 1)])
def test_results_compact_equal_full_records(kb, ctx, storage, flags):
    """kb_results_compact_async (16-byte records, pinned host and device destinations) carries
    the same values as kb_results, bit for bit: FP32 searches copy their device records as they
    are, rescored ones round the FP64 fields to FP32 as kb_results does for psi and phi."""
    st = synth.small_stack(92, 6, 70, 150, K=5, nan_frac=0.01, n_angles=8, n_speeds=8, s_hi=12.0, n_sources=3,
                           flux=40.0)
    N, H, W = st.sci.shape
    s = gpu_planes(kb, ctx, st, storage)
    job = kb.Job(ctx, H, W, N, st.vx.size, st.k, flags)
    job.search(s, st.times, st.vx, st.vy, st.k, -math.inf, flags)
    full = job.results()
    n = H * W * st.k * kb.COMPACT_DTYPE.itemsize
    pinned = torch.empty(n, dtype=torch.uint8, pin_memory=True)
    dev = torch.empty(n, dtype=torch.uint8, device=DEV)
    job.results_compact_async(pinned, stream=torch.cuda.Stream())
    job.results_compact_async(dev)
    torch.cuda.synchronize()
    got = pinned.numpy().view(kb.COMPACT_DTYPE)
    assert got.tobytes() == dev.cpu().numpy().tobytes()
    want = _compact_from_full(kb, full)
    for f in ("psi", "phi", "nu"):   # FP64 -> FP32 rounds to nearest on both sides
        assert np.array_equal(got[f].view(np.uint32), want[f].view(np.uint32)), f
    for f in ("vidx", "nobs", "reserved"):
        assert np.array_equal(got[f], want[f]), f
    with pytest.raises(kb.KBError):
        job.results_compact_async(np.empty(H * W * st.k, kb.COMPACT_DTYPE))
    with pytest.raises(kb.KBError):
        job.results_compact_async(torch.empty(n - 16, dtype=torch.uint8, device=DEV))
    job.free()
    s.free()


@pytest.mark.parametrize("cols", [1, 3, 5])
def test_tile_order_swizzle_equals_row_order(kb, ctx, cols):
    """kb_set_search_swizzle: tiles dealt out in super-columns (the last one narrower: 7 tile
    columns) give the row-order records byte for byte."""
    st = synth.small_stack(78, 4, 37, 7 * 64 - 5, K=3, n_angles=5, n_speeds=4, s_lo=5.0, s_hi=60.0, k=4)
    ref = gpu_search(kb, ctx, st)
    ctx.set_search_swizzle(cols)
    try:
        got = gpu_search(kb, ctx, st)
    finally:
        ctx.set_search_swizzle(-1)
    assert got.tobytes() == ref.tobytes()


@pytest.mark.parametrize("order", [1, 2])
def test_velocity_order_changes_no_result(kb, ctx, order):
    """kb_set_search_order: the Hilbert and the caller's velocity orders give the records of the
    default order byte for byte (ties in nu resolved by the caller's velocity index)."""
    st = synth.small_stack(79, 5, 60, 200, K=5, n_angles=9, n_speeds=7, s_lo=2.0, s_hi=40.0, k=8, n_sources=3,
                           flux=30.0)
    ref = gpu_search(kb, ctx, st)
    ctx.set_search_order(order)
    try:
        got = gpu_search(kb, ctx, st)
    finally:
        ctx.set_search_order(-1)
    assert got.tobytes() == ref.tobytes()
