"""Benchmark of the shift-and-stack likelihood search on GB300.

One step is one pass of the whole hot path over the DECam-shaped stack
(12 epochs of 4096 x 4096, 32 x 32 = 1024 velocities, k = 8):
psi/phi images (kb_make_psi_phi) and the exhaustive search (kb_search), plus
16-bit quantisation and FP64 rescoring when --storage bf16/f16 --rescore.
Metric: trajectory-epoch evaluations per second (H * W * V * N per step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--storage f32|bf16|f16] [--rescore]
                  [--impl ours|reference] [--size S]

--impl reference times the FP64 CPU oracle on the host cores instead (bounded
samples of start pixels of the same workload, whole path from the raw images).
Multi-GPU runs (torchrun) are independent replicas, one stack per GPU.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

# search-kernel algorithmic bytes per trajectory-epoch evaluation (one psi, phi pair)
BYTES_PER_EVAL = {"f32": 8, "bf16": 4, "f16": 4}

# The paper's own throughput for this metric (Sec. 2.3): about 2.4e-11 s per image per
# trajectory on 4K x 4K stacks, i.e. 4.2e10 trajectory-epoch evaluations per second, on an
# unnamed consumer GPU.  Another machine's number: context for vs_baseline, not a target.
PAPER_EVALS_PER_S = 4.2e10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--psf", default="gaussian", choices=["gaussian", "general"],
                    help="gaussian: the separable 17x17 Gaussians; general: rotated elliptical Gaussians "
                         "(not separable: the single-pass kernel over all K^2 taps)")
    ap.add_argument("--rescore", action="store_true")
    ap.add_argument("--size", type=int, default=4096, help="image side (4096 = the DECam workload)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--e2e-records", default="compact", choices=["compact", "full"],
                    help="records read back every end-to-end step: 16-byte kb_result_compact or 48-byte kb_result")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--variant", type=int, default=0, help="search kernel shape (0 = automatic)")
    ap.add_argument("--topk", type=int, default=0, help="results per pixel (0 = the workload's k)")
    ap.add_argument("--carveout", type=int, default=-1, help="search shared-memory carveout percent (-1 = auto)")
    ap.add_argument("--swizzle", type=int, default=-1, help="search tile order: super-columns of N tiles (-1 = auto)")
    ap.add_argument("--vorder", type=int, default=-1,
                    help="velocity order: 0 latest (dy, dx), 1 Hilbert, 2 the caller's (-1 = auto)")
    ap.add_argument("--workload", default="decam", choices=["decam", "batch", "serve"],
                    help="decam: the 12x4096^2 stack; batch: 64 uneven 2048x4096 stacks in one batched launch; "
                         "serve: a Poisson stream of search jobs through the serving loop")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--filter", action="store_true",
                    help="also time the Sec. 3.3 light-curve outlier filter on the kept trajectories")
    ap.add_argument("--stamps", type=int, default=0, metavar="M",
                    help="also time Sec. 3.3 coadded stamps (radius 10, mean and median, moments and cuts) of "
                         "the M highest-nu trajectories")
    ap.add_argument("--cluster", type=int, default=0, metavar="M",
                    help="also time Sec. 3.3 DBSCAN de-duplication of the M highest-nu trajectories")
    ap.add_argument("--threshold", type=float, default=0.0, metavar="NU_MIN",
                    help="also time the thresholded search (nu >= NU_MIN) with and without likelihood-bound "
                         "pruning (KB_PRUNE, Sec. 5.3); reported apart from the headline")
    ap.add_argument("--rp-steps", type=int, default=5,
                    help="default line: steps of the BF16 + FP64-rescoring leg beside the FP32 step (0 = off)")
    ap.add_argument("--serve-sample", type=int, default=150,
                    help="default line: jobs of the bounded serving sample with p50/p99 (0 = off)")
    ap.add_argument("--serve-jobs", type=int, default=2000)
    ap.add_argument("--serve-load", type=float, default=0.75,
                    help="arrival rate as a fraction of the capacity measured on a saturated sample")
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-policy", default="both", choices=["fifo", "sjf", "both"],
                    help="dispatch order of resident jobs: arrival order, least work first with aging, or "
                         "both in turn on the same arrivals (the line reports the last, sjf)")
    return ap.parse_args()


def dist_info():
    from paper_1901_02492_gb300 import replicas
    return replicas.dist_info()


def setup_device(world, local):
    """One process per GPU: bind this rank's device and join the (NCCL) group when N > 1."""
    import torch
    from paper_1901_02492_gb300 import replicas
    if world > 1:
        torch.cuda.set_device(local)
        replicas.init("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    return dev


def workload(size, psf="gaussian"):
    import synth
    st = synth.decam(H=size, W=size)
    if psf == "general":
        st.psf = synth.elongate_psfs(st.psf)       # rotated elliptical Gaussians: not separable
    return st


def roofline_psi_phi(args, st, ms, nbytes, hbm, clocks):
    """Stage (a) roofline.  Separable PSFs: HBM-bound (8 B read, 8 B written per pixel, more
    with 16-bit storage).  General PSFs: 2 K^2 FP32 FMAs per pixel (psi and phi) make it
    arithmetic-bound; the peak is 128 FP32 FMA lanes per SM x 2 FLOP x SM count x the SM clock
    sampled during the run."""
    import torch
    K = st.psf.shape[-1]
    stream = st.sci.shape[2] % 4 == 0 and 3 <= K <= 21   # the library's choice for separable PSFs
    line = {"bound": "hbm", "kernel": "psi_phi_stream_kernel" if stream else "psi_phi_sep_kernel", "ms_per_launch": ms,
            "achieved": nbytes / (ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
            "frac": nbytes / (ms * 1e-3) / 1e9 / hbm, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}
    if args.psf == "general":
        N, H, W = st.sci.shape
        K = st.psf.shape[-1]
        flops = 4.0 * N * H * W * K * K
        sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
        mhz = clocks.get("sm_mhz") or 2070.0
        peak = sms * 128 * 2 * mhz * 1e6 / 1e12
        tf = flops / (ms * 1e-3) / 1e12
        line = {"bound": "alu", "kernel": "psi_phi_gen_kernel<%d>" % K, "ms_per_launch": ms,
                "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                "flops_per_launch": flops,
                "peak_source": "derived: %d SMs x 128 FP32 lanes x 2 FLOP x %.0f MHz (sampled SM clock)" % (sms, mhz),
                "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm}
    return line


def workload_config(args, st, world):
    N, H, W = st.sci.shape
    name = "decam %dx%dx%d, %d velocities, k=%d" % (N, H, W, st.vx.size, st.k)
    return {"workload": name, "epochs": N, "height": H, "width": W, "velocities": int(st.vx.size),
            "topk": st.k, "psf": ("17x17 Gaussian, FWHM 3.5-4.5 px" if args.psf == "gaussian" else
                                  "17x17 rotated elliptical Gaussian, major FWHM 3.5-4.5 px, axis ratio "
                                  "0.6-0.9 (not separable)"), "storage": args.storage,
            "rescore_fp64": bool(args.rescore), "search_variant": args.variant, "carveout": args.carveout, "swizzle": args.swizzle,
            "velocity_order": args.vorder,
            "evals_per_step": int(N * H * W * st.vx.size),
            "l2": "inputs larger than L2 (%.2f GB of psi/phi planes)" % (N * H * W * 8 / 1e9),
            "parallelism": "replicas%d" % world}


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, gpu_index):
        import tempfile
        self.proc = None
        fd, self.path = tempfile.mkstemp(prefix="bench_clocks_", suffix=".csv")
        os.close(fd)
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        try:
            self.f.close()
        except Exception:
            pass

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    rows.append((float(parts[0]), float(parts[1]), float(parts[2]), parts[3:7]))
                except ValueError:
                    continue
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": reasons}


# ----------------------------------------------------------------------------- roofline helpers

def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def search_span(storage, variant, k):
    """Pixels per warp span of the register-gather search shape (the library's search_span)."""
    p32, p16 = [2, 4, 2, 4, 2], [2, 2, 1, 2, 1]
    v = variant if 1 <= variant <= 4 else 0
    if storage != "f32" and v == 0 and k > 8:
        return 64
    return 32 * p32[v] if storage == "f32" else 64 * p16[v]


def psf_moment_cuts(psf, aperture):
    """Moment-filter cuts from the epochs' PSFs: each PSF's per-axis second moment s^2 (of the
    sampled kernel), the second moment of that Gaussian inside the aperture, s^2 (1 - u e^-u /
    (1 - e^-u)) with u = aperture^2 / (2 s^2), averaged over epochs, plus 1/12 px^2 of pixel
    rounding; variances within [0.4, 1.8] of it, |mu11| within half of it, centroid within 1 px."""
    K = psf.shape[-1]
    c = np.arange(K) - K // 2
    w = psf.astype(np.float64)
    s2 = (w * (c[None, None, :] ** 2)).sum(axis=(1, 2)) / w.sum(axis=(1, 2))
    u = aperture ** 2 / (2.0 * s2)
    v0 = float(np.mean(s2 * (1.0 - u * np.exp(-u) / (1.0 - np.exp(-u))))) + 1.0 / 12.0
    return {"max_offset": 1.0, "min_var": 0.4 * v0, "max_var": 1.8 * v0, "max_mu11": 0.5 * v0}


def job_kkeep(k, rescore, storage):
    """Candidates per pixel the search keeps (the library's job_kkeep)."""
    if not rescore:
        return k
    return k + (max(2, k // 2) if storage == "bf16" else max(2, k // 4))


def recorded_levels(kernel_tag):
    """Per-level bytes of one search launch (L2 -> L1, DRAM) from the ncu summary in
    profiles/, scaled from the captured case to this workload by the gathered
    evaluations, when the kernel source is unchanged since (matching sha256 prefix)."""
    src = os.path.join(ROOT, "paper_1901_02492_gb300", "csrc", "kb_search.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    pdir = os.path.join(ROOT, "profiles")
    for fn in sorted(os.listdir(pdir)) if os.path.isdir(pdir) else []:
        if not fn.endswith(".md"):
            continue
        for line in open(os.path.join(pdir, fn)):
            m = re.match(r"levels\s+%s\s+(.*)\s+source_sha=([0-9a-f]+)$" % re.escape(kernel_tag), line.strip())
            if m and m.group(2) == sha:
                out = {"source": fn}
                for kv in m.group(1).split():
                    key, val = kv.split("=")
                    out[key] = float(val)
                return out
    return None


def recorded_traffic(kernel_tag):
    """DRAM bytes per launch recorded by an ncu capture in profiles/, if the kernel
    source has not changed since (matching sha256 prefix)."""
    src = os.path.join(ROOT, "paper_1901_02492_gb300", "csrc", "kb_search.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for fn in sorted(os.listdir(os.path.join(ROOT, "profiles"))) if os.path.isdir(os.path.join(ROOT, "profiles")) else []:
        if not fn.endswith(".md"):
            continue
        for line in open(os.path.join(ROOT, "profiles", fn)):
            m = re.match(r"traffic\s+%s\s+bytes_per_launch=(\d+)\s+source_sha=([0-9a-f]+)" % re.escape(kernel_tag),
                         line.strip())
            if m and m.group(2) == sha:
                return int(m.group(1))
    return None


def search_byte_classes(binding, times, vx, vy, H, W, bytes_per_eval, span):
    """The search's trajectory-epoch evaluations split by where their (psi, phi) pair
    comes from, counted on the host from the library's own offset table:
      ref      epochs at the reference time (offset 0 for every velocity): loaded once
               per start pixel, then reused for every velocity;
      off      trajectory pixel outside the image: nothing to gather (the kernel reads
               a zero block that stays in L1);
      gathered trajectory pixel inside the image: one pair gathered per evaluation.
    Algorithmic bytes per launch = gathered evaluations + one load per pixel and
    reference epoch, times the pair size.  `issued` counts what the kernel loads: whole
    warp spans of `span` pixels whose row is inside the image and whose columns overlap
    it (their off-image pixels read the zero columns beside every row)."""
    dx, dy = binding.offsets(times, vx, vy)              # [V][N], the caller's epoch order
    times = np.asarray(times, np.float64)
    V, N = dx.shape
    ref = (times == times.min()) & np.all(dx == 0, axis=0) & np.all(dy == 0, axis=0)
    nref = int(ref.sum())
    inx = np.maximum(0, W - np.abs(dx[:, ~ref])).astype(np.int64)
    iny = np.maximum(0, H - np.abs(dy[:, ~ref])).astype(np.int64)
    gathered = int((inx * iny).sum())
    total = H * W * V * N
    evals_ref = H * W * V * nref
    off = total - evals_ref - gathered
    # spans: tiles of `span` columns starting at multiples of span; overlap after the shift
    ntile = (W + span - 1) // span
    xs = np.arange(ntile, dtype=np.int64) * span
    issued = 0
    for v in range(V):
        for j in np.nonzero(~ref)[0]:
            ox, oy = int(dx[v, j]), int(dy[v, j])
            rows = max(0, H - abs(oy))
            if rows == 0:
                continue
            tiles = int(np.count_nonzero((xs + ox + span > 0) & (xs + ox < W)))
            issued += rows * tiles * span
    alg = (gathered + H * W * nref) * bytes_per_eval
    return {"evals_total": int(total), "evals_ref_epoch": int(evals_ref), "evals_off_image": int(off),
            "evals_gathered": gathered, "ref_epochs": nref,
            "alg_bytes_per_launch": int(alg),
            "issued_bytes_per_launch": int((issued + H * W * nref) * bytes_per_eval),
            "delivered_bytes_per_launch": int(total * bytes_per_eval)}


# ----------------------------------------------------------------------------- reference arm (oracle)

def oracle_sample(st, seconds, rng):
    """Time the oracle's whole path (psi/phi from the raw images + search) on a bounded
    sample of start pixels of the workload; returns (evals, seconds, pixels)."""
    import oracle
    N, H, W = st.sci.shape
    dx, dy = oracle.offsets(st.times, st.vx, st.vy)
    n = max(1, oracle.num_threads())
    done, spent = 0, 0.0
    while spent < min(0.5, seconds / 4):        # calibrate on at least 0.5 s of work
        m = n * max(1, 2 ** min(done // n, 6))
        px = rng.integers(0, W, m)
        py = rng.integers(0, H, m)
        t0 = time.perf_counter()
        oracle.search_pixels_from_images(st.sci, st.var, None, st.psf, st.times, dx, dy, st.k, px, py)
        spent += time.perf_counter() - t0
        done += m
    per_pix = spent / done
    npix = max(n, int(seconds / max(per_pix, 1e-9)) // n * n)
    px = rng.integers(0, W, npix)
    py = rng.integers(0, H, npix)
    t0 = time.perf_counter()
    oracle.search_pixels_from_images(st.sci, st.var, None, st.psf, st.times, dx, dy, st.k, px, py)
    dt = time.perf_counter() - t0
    return npix * st.vx.size * N, dt, npix


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import oracle
    st = workload(args.size, args.psf)
    cfg = workload_config(args, st, 1)
    rng = np.random.default_rng(1234)
    per_step = max(2.0, min(10.0, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(st, per_step / 4, rng)
    evals = 0
    secs = 0.0
    pix = 0
    for _ in range(args.steps):
        e, s, p = oracle_sample(st, per_step, rng)
        evals += e
        secs += s
        pix += p
    value = evals / secs
    line = {"impl": "reference", "metric": "trajectory-epoch evals/sec on 12x4096^2 stack",
            "value": value, "unit": "evals/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * secs / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "evals/s", "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": "%d random start pixels x %d velocities x %d epochs of the workload, "
                                       "psi/phi evaluated from the raw images" % (pix, st.vx.size, st.sci.shape[0])},
            "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    from paper_1901_02492_gb300 import replicas
    rank, world, local = dist_info()
    dev = setup_device(world, local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1901_02492_gb300 import binding as kb

    st = workload(args.size, args.psf)
    N, H, W = st.sci.shape
    V = st.vx.size
    if args.topk:
        st.k = args.topk
    k = st.k
    evals = N * H * W * V
    flags = kb.KB_RESCORE_FP64 if args.rescore else 0
    ctx = kb.Context(dev.index)
    ctx.set_search_variant(args.variant)
    ctx.set_search_carveout(args.carveout)
    ctx.set_search_swizzle(args.swizzle)
    ctx.set_search_order(args.vorder)
    stack = kb.Stack(ctx, N, H, W, args.storage)
    job = kb.Job(ctx, H, W, N, V, k, flags)
    sci_h = torch.from_numpy(st.sci).pin_memory()
    var_h = torch.from_numpy(st.var).pin_memory()
    sci = sci_h.to(dev)
    var = var_h.to(dev)
    stream = torch.cuda.current_stream(dev)
    # roofline denominators, before the timed region: the L2-to-SM rate of the search's own
    # access form (the warp span of the launch shape, 512 B for the default shapes, at any 8-byte offset),
    # and of line-aligned spans for reference
    span = search_span(args.storage, args.variant, job_kkeep(k, args.rescore, args.storage))
    span_bytes = span * BYTES_PER_EVAL[args.storage]
    gather_peak = ctx.measure_gather_peak(span_bytes, 8)
    gather_peak_aligned = ctx.measure_gather_peak(span_bytes, 256)
    launches_per_step = 2 + (1 if args.storage != "f32" else 0) + (2 if args.rescore else 0)

    ev = lambda: torch.cuda.Event(enable_timing=True)

    def step(timers=None):
        if timers is not None:
            timers[0].record(stream)
        stack.make_psi_phi(sci, var, None, st.psf, stream=stream)
        if timers is not None:
            timers[1].record(stream)
        job.search(stack, st.times, st.vx, st.vy, k, -math.inf, flags, stream=stream)
        if timers is not None:
            timers[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    replicas.barrier()
    torch.cuda.synchronize(dev)
    timers = [[ev(), ev(), ev()] for _ in range(args.steps)]
    with ClockSampler(dev.index) as clk:
        t0, t1 = ev(), ev()
        t0.record(stream)
        for i in range(args.steps):
            step(timers[i])
        t1.record(stream)
        torch.cuda.synchronize(dev)
    replicas.barrier()
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    repaired = job.repaired() if args.rescore else 0
    ms_psiphi = sum(t[0].elapsed_time(t[1]) for t in timers) / args.steps
    ms_search = sum(t[1].elapsed_time(t[2]) for t in timers) / args.steps
    clocks = clk.summary()

    # End to end through the C ABI, every step: pinned host inputs -> device -> psi/phi ->
    # search -> all H*W*k records to pinned host memory.  Steps are pipelined over three
    # streams: step i+1's inputs go up (s_in) and step i's records come back (s_out, with
    # kb_results_async) while the GPU computes; inputs and jobs are double-buffered.
    rec_dtype = kb.COMPACT_DTYPE if args.e2e_records == "compact" else kb.RESULT_DTYPE
    nrec_bytes = H * W * k * rec_dtype.itemsize
    res_h = [torch.empty(nrec_bytes, dtype=torch.uint8, pin_memory=True) for _ in range(2)]
    jobs = [job, kb.Job(ctx, H, W, N, V, k, flags)]
    sci_d, var_d = [sci, torch.empty_like(sci)], [var, torch.empty_like(var)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_psi = [torch.cuda.Event() for _ in range(2)]

    comp_ev = []

    def e2e_step(i, timed=False):
        b = i % 2
        s_in.wait_event(ev_psi[b])                 # psi/phi of step i-2 has read buffer b
        with torch.cuda.stream(s_in):
            sci_d[b].copy_(sci_h, non_blocking=True)
            var_d[b].copy_(var_h, non_blocking=True)
        ev_in[b].record(s_in)
        stream.wait_event(ev_in[b])
        if timed:
            comp_ev.append((ev(), ev()))
            comp_ev[-1][0].record(stream)
        stack.make_psi_phi(sci_d[b], var_d[b], None, st.psf, stream=stream)
        ev_psi[b].record(stream)
        # waits (on the device) for the read of this job's step i-2 records
        jobs[b].search(stack, st.times, st.vx, st.vy, k, -math.inf, flags, stream=stream)
        if timed:
            comp_ev[-1][1].record(stream)
        if args.e2e_records == "compact":
            jobs[b].results_compact_async(res_h[b], stream=s_out)
        else:
            jobs[b].results_async(res_h[b], stream=s_out)

    n_e2e = max(args.e2e_steps, 2)
    for i in range(2):
        e2e_step(i)
    torch.cuda.synchronize(dev)
    a = time.perf_counter()
    for i in range(2, 2 + n_e2e):
        e2e_step(i, timed=True)
    torch.cuda.synchronize(dev)
    e2e_ms = 1e3 * (time.perf_counter() - a) / n_e2e
    # device time of psi/phi + search inside the pipeline (beside the copies)
    e2e_comp_ms = float(np.mean([t0.elapsed_time(t1) for t0, t1 in comp_ev]))
    for j in jobs:
        j.wait()
    if args.e2e_records == "compact" and (args.stamps > 0 or args.cluster > 0):
        res_np = job.results()      # full records of the last search, for the post-search legs
    elif args.e2e_records != "compact":
        res_np = res_h[(1 + n_e2e) % 2].numpy().view(kb.RESULT_DTYPE)   # the last step's records

    # the slowest rank's times (replicas: every rank searched its own copy of the stack)
    ms, e2e_ms = replicas.max_over_ranks([ms, e2e_ms], device=dev)
    value = world * evals * args.steps / (ms * 1e-3)
    peaks = measured_peaks()

    # Roofline of the dominant kernel, the search.  Algorithmic bytes: one (psi, phi)
    # pair per trajectory-epoch evaluation (8 B in FP32, 4 B in 16-bit storage).  The
    # gathers are served by L2 (L1 catches the early epochs' reuse, HBM sees little:
    # the planes stay L2-resident), so the denominator is the L2-to-SM bandwidth of
    # exactly this access form, measured on this device by the library.
    classes = search_byte_classes(kb, st.times, st.vx, st.vy, H, W, BYTES_PER_EVAL[args.storage], span)
    alg_bytes = classes["alg_bytes_per_launch"]
    achieved = alg_bytes / (ms_search * 1e-3) / 1e9
    delivered = classes["delivered_bytes_per_launch"] / (ms_search * 1e-3) / 1e9
    # the captured counters belong to the value-list search kernels; a rescored search runs the
    # key-list kernel and the rescoring kernels inside the timed call, which have none recorded
    tag = "search_%s%s" % (args.storage, "_rescored" if args.rescore else "")
    traffic = recorded_traffic(tag)
    levels = recorded_levels(tag)
    if levels and "l2_to_l1_bytes_per_alg_byte" in levels:
        # the L2 -> SM share at this size: the captured ratio to the algorithmic bytes
        l2b = levels["l2_to_l1_bytes_per_alg_byte"] * alg_bytes
        levels["l2_to_l1_bytes_per_launch"] = l2b
        levels["l2_to_l1_GBps"] = l2b / (ms_search * 1e-3) / 1e9
        levels["l2_to_l1_frac"] = levels["l2_to_l1_GBps"] / gather_peak
    hbm = peaks.get("hbm_gbs", 6800.0)
    psiphi_bytes = N * H * W * (8 + 8 + (4 + 8 if args.storage != "f32" else 0))
    cfg = workload_config(args, st, world)
    line = {"metric": "trajectory-epoch evals/sec on 12x4096^2 stack", "value": value, "unit": "evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_EVALS_PER_S,
            "vs_baseline_note": "value / 4.2e10 evals/s, the paper's figure on its own (unnamed consumer) GPU",
            "dtype": args.storage, "data": "synthetic", "config": cfg,
            "roofline": {"bound": "l2",
                         "kernel": ("kb_search call: search_kernel (key lists) + rescore_kernel + repair_kernel"
                                    if args.rescore else "search_kernel"),
                         "achieved": achieved, "peak": gather_peak,
                         "unit": "GB/s", "frac": achieved / gather_peak, "traffic": traffic,
                         "peak_source": "measured in this run by kb_measure_gather_peak(%d, 8): L2-resident "
                                        "%d-byte warp spans at any 8-byte offset (the search's access form), "
                                        "not cached in L1" % (span_bytes, span_bytes),
                         "ms_per_launch": ms_search, "alg_bytes_per_launch": alg_bytes,
                         "alg_bytes_note": "gathered (in-image, non-reference-epoch) evaluations + one load per "
                                           "pixel and reference epoch, x %d B" % BYTES_PER_EVAL[args.storage],
                         "byte_classes": classes,
                         "frac_issued": classes["issued_bytes_per_launch"] / (ms_search * 1e-3) / 1e9 / gather_peak,
                         "frac_delivered": delivered / gather_peak,
                         "frac_delivered_note": "every trajectory-epoch evaluation counted as a gather (the "
                                                "figure an evals/s rate implies)",
                         "peak_aligned_spans": gather_peak_aligned,
                         "levels": levels},
            "roofline_psi_phi": roofline_psi_phi(args, st, ms_psiphi, psiphi_bytes, hbm, clocks),
            "clocks": clocks,
            "e2e": {"value": world * evals / (e2e_ms * 1e-3), "unit": "evals/s",
                    "h2d_bytes_per_step": int(sci_h.numel() * 4 + var_h.numel() * 4),
                    "d2h_bytes_per_step": int(nrec_bytes), "ms_per_step": e2e_ms,
                    "steps": n_e2e, "compute_ms_per_step": e2e_comp_ms,
                    "records": "%s (%d B each, all H*W*k every step)" % (args.e2e_records, rec_dtype.itemsize),
                    "pipeline": "host clock over %d steps; inputs and jobs double-buffered, uploads, "
                                "compute and %s reads on three streams"
                                % (n_e2e, "kb_results_compact_async" if args.e2e_records == "compact"
                                   else "kb_results_async")},
            "gpu_launches": launches_per_step * args.steps}
    if args.threshold > 0:
        # the thresholded search (Sec. 5.2's nu_min), plain and with likelihood-bound pruning: the
        # same records, the pruned one skipping the gathers of spans whose bound is below nu_min
        nu_min = float(args.threshold)
        tout = [torch.empty(H * W * k * kb.COMPACT_DTYPE.itemsize, dtype=torch.uint8, device=dev) for _ in range(2)]
        tms = {}
        for i, (name, fl) in enumerate((("plain", flags), ("pruned", flags | kb.KB_PRUNE))):
            job.search(stack, st.times, st.vx, st.vy, k, nu_min, fl, stream=stream)   # warm-up (builds the bounds)
            t0, t1 = ev(), ev()
            t0.record(stream)
            for _ in range(3):
                job.search(stack, st.times, st.vx, st.vy, k, nu_min, fl, stream=stream)
            t1.record(stream)
            job.results_compact_async(tout[i], stream=stream)
            torch.cuda.synchronize(dev)
            tms[name] = t0.elapsed_time(t1) / 3
        kept = int((tout[1].view(torch.int32).view(-1, 4)[:, 3] & 0xFFFF != 0xFFFF).sum().item())
        line["thresholded"] = {"nu_min": nu_min, "ms_per_search_plain": tms["plain"],
                               "ms_per_search_pruned": tms["pruned"], "speedup": tms["plain"] / tms["pruned"],
                               "records_identical": bool(torch.equal(tout[0], tout[1])), "kept_trajectories": kept,
                               "nominal_evals_per_s_pruned": evals / (tms["pruned"] * 1e-3),
                               "note": "nominal: every trajectory-epoch evaluation of the grid, skipped ones included"}
        del tout
    if args.filter:
        # the Sec. 3.3 outlier filter of every kept trajectory (two FP64 passes over its epochs)
        fout = torch.empty(H * W * k * kb.FILTERED_DTYPE.itemsize, dtype=torch.uint8, device=dev)
        job.filter_lightcurves(stack, 5.0, fout, stream=stream)
        f0, f1 = ev(), ev()
        f0.record(stream)
        for _ in range(3):
            job.filter_lightcurves(stack, 5.0, fout, stream=stream)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        fms = f0.elapsed_time(f1) / 3
        nrej = int(fout.view(torch.int32).view(H * W * k, kb.FILTERED_DTYPE.itemsize // 4)[:, 4].sum().item())
        line["filter"] = {"kernel": "filter_kernel", "nsigma": 5.0, "ms_per_launch": fms,
                          "trajectories_per_s": H * W * k / (fms * 1e-3), "rejected_epochs": nrej,
                          "trajectories": H * W * k}
        del fout
    if args.stamps > 0:
        # Sec. 3.3 coadded stamps of the M best trajectories of the last search (21 x 21, every epoch),
        # moments over a 3 px aperture, cuts from the epochs' PSF widths
        M, r, ap = args.stamps, 10, 3.0
        flat = res_np.reshape(-1)
        best = np.argpartition(-np.where(flat["vidx"] >= 0, flat["nu"], -np.inf), M - 1)[:M]
        cx, cy, cv = flat["x0"][best].copy(), flat["y0"][best].copy(), flat["vidx"][best].copy()
        cuts = psf_moment_cuts(st.psf, ap)
        # candidates on an injected source: start within 3 px of it and velocity within 40 px/day
        near = np.zeros(M, bool)
        hit = set()
        for si, src in enumerate(st.sources):
            m = ((np.abs(cx - src["x0"]) <= 3.0) & (np.abs(cy - src["y0"]) <= 3.0) &
                 (np.hypot(st.vx[cv] - src["vx"], st.vy[cv] - src["vy"]) <= 40.0))
            near |= m
            if m.any():
                hit.add(si)
        line["stamps"] = {"kernel": "stamp_kernel", "candidates": M, "radius": r, "aperture_px": ap, "cuts": cuts,
                          "candidates_on_injected_sources": int(near.sum()), "injected_sources_hit": len(hit),
                          "injected_sources": len(st.sources)}
        S2 = (2 * r + 1) ** 2
        for mode in ("mean", "median"):
            job.stamps(sci, None, cx, cy, cv, r, median=mode == "median", cuts=cuts, stream=stream, aperture=ap)
            s0, s1 = ev(), ev()
            s0.record(stream)
            for _ in range(3):
                _, mom = job.stamps(sci, None, cx, cy, cv, r, median=mode == "median", cuts=cuts, stream=stream,
                                    aperture=ap)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            sms = s0.elapsed_time(s1) / 3
            gathered = M * S2 * N * 4 + M * S2 * 4
            passed = mom["passed"].astype(bool)
            line["stamps"][mode] = {"ms_per_call": sms, "stamps_per_s": M / (sms * 1e-3),
                                    "gathered_GBps": gathered / (sms * 1e-3) / 1e9,
                                    "passed_cuts": int(passed.sum()),
                                    "pass_rate_on_injected_sources": float(passed[near].mean()) if near.any() else None,
                                    "pass_rate_rest": float(passed[~near].mean())}
    if args.cluster > 0:
        # Sec. 3.3 DBSCAN de-duplication of the M best trajectories of the last search: 2 px and
        # 15 px/day (about half the velocity grid's radial step) per unit, eps 1.5, min_samples 4
        M = args.cluster
        flat = res_np.reshape(-1)
        best = np.sort(np.argpartition(-np.where(flat["vidx"] >= 0, flat["nu"], -np.inf), M - 1)[:M])
        cand = torch.from_numpy(flat[best].view(np.uint8).copy()).to(dev)
        prm = dict(w_pos=0.5, w_vel=1.0 / 15.0, eps=1.5, min_samples=4)
        ctx.cluster(cand, stream=stream, **prm)
        c0, c1 = ev(), ev()
        c0.record(stream)
        for _ in range(3):
            _, keep, _, groups = ctx.cluster(cand, stream=stream, **prm)
        c1.record(stream)
        torch.cuda.synchronize(dev)
        cms = c0.elapsed_time(c1) / 3
        line["cluster"] = {"kernels": "kb_cluster (8 launches)", "candidates": M, "params": prm,
                           "ms_per_call": cms, "candidates_per_s": M / (cms * 1e-3), "groups": groups}
        del cand
    if args.rescore:
        line["rescore"] = {"candidates_per_pixel": job_kkeep(k, True, args.storage),
                           "repaired_pixels": repaired,
                           "repaired_fraction": repaired / float(H * W)}
    if world == 1 and args.rp_steps > 0 and args.storage == "f32" and not args.rescore:
        line["reduced_precision"] = reduced_precision_leg(args, kb, ctx, st, sci, var, stream, dev, jobs[0],
                                                          ms / args.steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        e, s, p = oracle_sample(st, args.cpu_seconds, np.random.default_rng(7))
        line["cpu_baseline"] = {"value": e / s, "unit": "evals/s", "cores": oracle.num_threads(), "kind": "oracle",
                                "sample": "%d random start pixels x %d velocities x %d epochs of the workload, "
                                          "psi/phi evaluated from the raw images, %.1f s" % (p, V, N, s)}
    for j in jobs:
        j.free()
    stack.free()
    ctx.close()
    del sci, var, sci_d, var_d, res_h
    torch.cuda.empty_cache()
    if world == 1 and args.serve_sample > 0 and args.size == 4096:
        line["serving_sample"] = serving_sample_leg(args, dev, kb)
    if rank == 0:
        print(json.dumps(line), flush=True)
    replicas.finish()


def reduced_precision_leg(args, kb, ctx, st, sci, var, stream, dev, job32, ms_fp32):
    """The same stack and grid with BF16 planes (per-epoch power-of-two scales) and the top-k
    rescored in FP64 from the FP32 planes: ms per step (psi/phi, quantize, candidate search,
    rescoring, repair) against the FP32 step just timed, and the slots whose velocity index equals
    the FP32 path's (they differ only at near-ties of the FP32 search, which the FP64 oracle
    decides: the rescored top-k is the oracle's, see the precision tests)."""
    import torch
    N, H, W = st.sci.shape
    V, k = st.vx.size, st.k
    flags = kb.KB_RESCORE_FP64
    stack = kb.Stack(ctx, N, H, W, "bf16")
    job = kb.Job(ctx, H, W, N, V, k, flags)

    def step():
        stack.make_psi_phi(sci, var, None, st.psf, stream=stream)
        job.search(stack, st.times, st.vx, st.vy, k, -math.inf, flags, stream=stream)

    for _ in range(2):
        step()
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.rp_steps):
        step()
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1) / args.rp_steps
    nrec = H * W * k
    a = torch.empty(nrec * kb.COMPACT_DTYPE.itemsize, dtype=torch.uint8, device=dev)
    b = torch.empty_like(a)
    job32.results_compact_async(a, stream=stream)
    job.results_compact_async(b, stream=stream)
    torch.cuda.synchronize(dev)
    ra, rb = a.view(torch.int32).view(nrec, 4), b.view(torch.int32).view(nrec, 4)
    same = (ra[:, 3] & 0xFFFF) == (rb[:, 3] & 0xFFFF)
    nu_a, nu_b = ra[:, 2].view(torch.float32)[same], rb[:, 2].view(torch.float32)[same]
    rel = ((nu_a - nu_b).abs() / nu_b.abs().clamp(min=1.0)).max().item() if bool(same.any()) else None
    out = {"storage": "bf16", "rescore_fp64": True, "steps": args.rp_steps, "ms_per_step": ms,
           "evals_per_s": N * H * W * V / (ms * 1e-3), "fp32_ms_per_step": ms_fp32,
           "speed_vs_fp32_step": ms_fp32 / ms,
           "candidates_per_pixel": job_kkeep(k, True, "bf16"), "repaired_pixels": job.repaired(),
           "slots_equal_to_fp32": float(same.float().mean().item()),
           "nu_max_rel_diff_vs_fp32_on_equal_slots": rel,
           "timing": "CUDA events over %d steps after 2 warm-up steps, inputs resident" % args.rp_steps}
    del a, b, ra, rb
    job.free()
    stack.free()
    return out


def serving_sample_leg(args, dev, kb):
    """A bounded sample of the serving workload for the default line: the first
    `--serve-sample` jobs of the serving stream, FIFO dispatch at `--serve-load` of the capacity
    measured on a saturated sample of 60 of them, p50/p99 latency beside the serial plain-FP32
    loop on the same arrivals (`--workload serve` runs the whole 2,000-job stream)."""
    r = serve_measure(args, dev, kb, args.serve_sample, 60, ["fifo"])
    lat, ser_lat, svc = r["lat"], r["ser_lat"], r["svc"]
    pct = lambda x, q: float(np.percentile(x, q))
    return {"jobs": len(r["done"]), "policy": "fifo", "slots": args.serve_slots,
            "hbm_budget_gb": args.serve_budget_gb, "arrival_rate_hz": r["rate"], "capacity_jobs_s": r["cap_jobs_s"],
            "served_bf16_rescored": {"p50_s": pct(lat, 50), "p99_s": pct(lat, 99), "mean_s": float(lat.mean()),
                                     "jobs_per_s": len(r["done"]) / r["wall"],
                                     "gpu_busy_fraction": r["main"]["busy"]},
            "serial_fp32": {"p50_s": pct(ser_lat, 50), "p99_s": pct(ser_lat, 99),
                            "capacity_jobs_s": len(r["reqs"]) / float(svc.sum())},
            "capacity_vs_serial_fp32": r["cap_jobs_s"] / (len(r["reqs"]) / float(svc.sum())),
            "clocks": r["main"]["clocks"],
            "note": "sample of the serving workload's job stream; p99 over this many jobs is near its maximum"}


def run_batch(args):
    """The uneven batch: 64 stacks (W 2048 x H 4096, 5-20 epochs, 256-2048 velocities, k 4-16)
    searched by one graph-captured persistent launch per storage group (kb_batch_run), tile
    shape chosen by the library's autotuner.  One step = one kb_batch_run over all stacks.
    Beside it: the same searches as a loop of single kb_search calls."""
    import torch
    import synth
    from paper_1901_02492_gb300 import replicas
    rank, world, local = dist_info()
    dev = setup_device(world, local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1901_02492_gb300 import binding as kb

    H, W = 4096, 2048
    specs = synth.batch_specs(count=args.batch_count)
    flags = kb.KB_RESCORE_FP64 if args.rescore else 0
    ctx = kb.Context(dev.index)
    ctx.set_search_carveout(args.carveout)
    stream = torch.cuda.current_stream(dev)
    stacks, jobs, searches, evals = [], [], [], 0
    t_gen = time.perf_counter()
    for sp in specs:
        times, psf, vx, vy, k = synth.batch_meta(sp)
        N = sp["N"]
        sci, var = synth.images_device(sp["seed"], N, H, W, dev)
        s = kb.Stack(ctx, N, H, W, args.storage)
        s.make_psi_phi(sci, var, None, psf, stream=stream)
        torch.cuda.synchronize(dev)
        del sci, var
        j = kb.Job(ctx, H, W, N, vx.size, k, flags)
        stacks.append(s)
        jobs.append(j)
        searches.append(dict(job=j, stack=s, times=times, vx=vx, vy=vy, topk=k, flags=flags))
        evals += N * H * W * vx.size
    t_gen = time.perf_counter() - t_gen
    torch.cuda.empty_cache()

    # the same searches one kb_search call at a time (the plain single-stack path)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    for d in searches[:2]:
        d["job"].search(d["stack"], d["times"], d["vx"], d["vy"], d["topk"], -math.inf, flags, stream=stream)
    torch.cuda.synchronize(dev)
    a, b = ev(), ev()
    a.record(stream)
    for d in searches:
        d["job"].search(d["stack"], d["times"], d["vx"], d["vy"], d["topk"], -math.inf, flags, stream=stream)
    b.record(stream)
    torch.cuda.synchronize(dev)
    ms_loop = a.elapsed_time(b)

    t_tune = time.perf_counter()
    batch = kb.Batch(ctx, searches, autotune=True)
    t_tune = time.perf_counter() - t_tune
    groups = batch.groups()
    gather_peak = ctx.measure_gather_peak(512 if args.storage == "f32" else 256, 8)
    for _ in range(args.warmup):
        batch.run(stream)
    torch.cuda.synchronize(dev)
    replicas.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index) as clk:
        t0, t1 = ev(), ev()
        t0.record(stream)
        for _ in range(args.steps):
            batch.run(stream)
        t1.record(stream)
        torch.cuda.synchronize(dev)
    replicas.barrier()
    torch.cuda.synchronize(dev)
    ms = t0.elapsed_time(t1)
    ms = replicas.max_over_ranks([ms], device=dev)[0]
    value = world * evals * args.steps / (ms * 1e-3)
    alg_bytes = evals * BYTES_PER_EVAL[args.storage]
    achieved = alg_bytes / (ms / args.steps * 1e-3) / 1e9
    # kernels per kb_batch_run: one per persistent group, one per search of a launch group, and the
    # rescore + repair kernels of each rescored search (groups: searches with the same list length)
    kkeep = [d["topk"] if not flags else None for d in searches]
    launches_per_run = sum(1 if g.schedule == 0 else sum(1 for kk in kkeep if kk == g.kmax) for g in groups)
    launches_per_run += 2 * len(searches) if flags else 0
    cfg = {"workload": "batch of %d uneven stacks, W %d x H %d, 5-20 epochs, 256-2048 velocities, k 4-16"
                       % (len(specs), W, H),
           "stacks": len(specs), "height": H, "width": W, "epochs_total": int(sum(sp["N"] for sp in specs)),
           "evals_per_step": int(evals), "storage": args.storage, "rescore_fp64": bool(args.rescore),
           "groups": [{"storage": g.storage, "variant": g.variant, "schedule": ["persistent", "launches"][g.schedule],
                       "index_bits": g.index_bits, "kmax": g.kmax, "items": int(g.n_items),
                       "tuned_ms_persistent": [round(x, 3) for x in list(g.tuned_ms)[1:]],
                       "tuned_ms_launches": [round(x, 3) for x in list(g.tuned_ms_launch)[1:]]}
                      for g in groups],
           "autotune_s": round(t_tune, 3), "generate_s": round(t_gen, 1),
           "l2": "inputs larger than L2 (%.1f GB of psi/phi planes)" % (sum(sp["N"] for sp in specs) * H * W * 8 / 1e9),
           "inputs": "drawn on the device (torch Philox), noise and mask model of the DECam stack",
           "parallelism": "replicas%d" % world}
    line = {"metric": "trajectory-epoch evals/sec, batched uneven stacks", "value": value, "unit": "evals/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
            "data": "synthetic", "config": cfg,
            "single_search_loop": {"value": world * evals / (ms_loop * 1e-3), "unit": "evals/s", "ms": ms_loop},
            "roofline": {"bound": "l2", "kernel": "search_batch_kernel", "achieved": achieved, "peak": gather_peak,
                         "unit": "GB/s", "frac": achieved / gather_peak, "traffic": None,
                         "peak_source": "measured in this run by kb_measure_gather_peak (the search's span form)",
                         "frac_note": "every trajectory-epoch evaluation counted as a gather (delivered)"},
            "clocks": clk.summary(), "e2e": None,
            "e2e_note": "inputs of the 64 stacks are drawn on the device; the end-to-end number is on the "
                        "single-stack line",
            "gpu_launches": args.steps * launches_per_run}
    if rank == 0:
        print(json.dumps(line), flush=True)
    batch.free()
    for j in jobs:
        j.free()
    for s in stacks:
        s.free()
    ctx.close()
    replicas.finish()


def run_serve(args):
    """The serving workload: Poisson arrivals of search jobs of 512^2, 4096 x 2048 and 4096^2
    pixels, 5-15 epochs, 256-1024 velocities, k = 8, BF16 planes with FP64 rescoring, admitted
    under an HBM budget and overlapped on `--serve-slots` streams.  The arrival rate is set to
    `--serve-load` of the loop's measured capacity.  Beside it, the plain FP32 serial loop: each
    job alone (upload, psi/phi, FP32 search, results to the host), its measured service times
    queued first-come first-served on the same arrival times."""
    from paper_1901_02492_gb300 import replicas
    rank, world, local = dist_info()
    dev = setup_device(world, local)
    import __graft_entry__
    __graft_entry__.build()
    from paper_1901_02492_gb300 import binding as kb

    r = serve_measure(args, dev, kb, args.serve_jobs, 300, ["fifo", "sjf"] if args.serve_policy == "both"
                      else [args.serve_policy])
    policies, jobs, done, wall, lat = r["policies"], r["jobs"], r["done"], r["wall"], r["lat"]
    main, served, evals, reqs, svc, ser_lat = r["main"], r["served"], r["evals"], r["reqs"], r["svc"], r["ser_lat"]
    total_evals = sum(evals[c.id] for c in done)

    def pct(x, q):
        return float(np.percentile(x, q))

    line = {"metric": "serving: p50/p99 job latency and throughput vs a serial plain-FP32 loop",
            "value": total_evals / wall, "unit": "evals/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": wall * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16", "data": "synthetic",
            "config": {"workload": "serving: %d Poisson-arrival jobs of 512^2, 4096x2048, 4096^2 px, 5-15 epochs, "
                                   "256-1024 velocities, k=8, BF16 + FP64 rescoring" % len(jobs),
                       "jobs": len(jobs), "slots": args.serve_slots, "hbm_budget_gb": args.serve_budget_gb,
                       "dispatch_policy": policies[-1],
                       "arrival_rate_hz": r["rate"], "capacity_jobs_s": r["cap_jobs_s"],
                       "target_load": args.serve_load,
                       "inputs": "pinned host stacks per size class (drawn on the device), copied to the device "
                                 "per job", "generate_s": round(r["t_gen"], 1), "parallelism": "replicas%d" % world},
            "serving": {"p50_s": pct(lat, 50), "p99_s": pct(lat, 99), "mean_s": float(lat.mean()),
                        "jobs_per_s": len(done) / wall, "gpu_busy_fraction": main["busy"],
                        "peak_device_bytes": int(main["peak"])},
            "serving_by_policy": {pol: {"p50_s": pct(v["lat"], 50), "p99_s": pct(v["lat"], 99),
                                        "mean_s": float(v["lat"].mean()), "jobs_per_s": len(v["done"]) / v["wall"],
                                        "gpu_busy_fraction": v["busy"]} for pol, v in served.items()},
            "serial_fp32": {"p50_s": pct(ser_lat, 50), "p99_s": pct(ser_lat, 99),
                            "jobs_per_s": len(reqs) / float(svc.sum()),
                            "evals_per_s": sum(evals.values()) / float(svc.sum()),
                            "mean_service_s": float(svc.mean())},
            "clocks": main["clocks"],
            "e2e": {"value": total_evals / wall, "unit": "evals/s",
                    "h2d_bytes_per_step": int(sum(2 * 4 * jobs[c.id]["N"] * jobs[c.id]["H"] * jobs[c.id]["W"]
                                                  for c in done)),
                    "d2h_bytes_per_step": int(sum(48 * 8 * jobs[c.id]["H"] * jobs[c.id]["W"] for c in done))},
            # per job: psi/phi, quantize, search, rescore, repair, expand (results to the device buffer)
            "gpu_launches": 6 * len(done)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    replicas.finish()


def serve_measure(args, dev, kb, n_jobs, n_calib, policies):
    """Serving measurement shared by the serve workload and the default line's sample: the first
    n_jobs jobs of the serving stream (BF16 + FP64 rescoring, `--serve-slots` slots, the HBM
    budget), arriving at `--serve-load` of the capacity measured on a saturated sample of n_calib
    jobs, under each dispatch policy in turn; then the serial plain-FP32 loop's service times, queued
    first-come first-served on the same arrivals.  Uses a context of its own (the budget)."""
    import torch
    import synth
    from paper_1901_02492_gb300 import serve

    budget = int(args.serve_budget_gb * 1e9)
    ctx = kb.Context(dev.index, budget)
    t_gen = time.perf_counter()
    jobs = synth.serving_jobs(count=n_jobs, rate_hz=1.0)
    max_n = max(j["N"] for j in jobs)
    pools = {}
    for (H, W) in sorted({(j["H"], j["W"]) for j in jobs}):
        sci, var = synth.images_device(1000 + H + W, max_n, H, W, dev)
        pools[(H, W)] = (sci.cpu().pin_memory(), var.cpu().pin_memory())
        del sci, var
    torch.cuda.empty_cache()
    metas = [synth.serving_meta(j) for j in jobs]

    def requests(rate, which=None):
        idx = range(len(jobs)) if which is None else which
        out = []
        for i in idx:
            j, (times, psf, vx, vy, k) = jobs[i], metas[i]
            sci, var = pools[(j["H"], j["W"])]
            payload = dict(sci=sci, var=var, psf=psf, times=times, vx=vx, vy=vy)
            arr = 0.0 if rate is None else j["arrival"] / rate
            out.append(serve.Request(i, arr, j["N"], j["H"], j["W"], psf.shape[-1], vx.size, k, payload))
        return out

    max_npix = max(j["H"] * j["W"] for j in jobs)
    max_planes = max_n * max_npix
    evals = {i: jobs[i]["N"] * jobs[i]["H"] * jobs[i]["W"] * metas[i][2].size for i in range(len(jobs))}
    t_gen = time.perf_counter() - t_gen

    def backend(storage, rescore, slots):
        return serve.CudaBackend(ctx, dev, storage=storage, rescore=rescore, slots=slots, max_npix=max_npix,
                                 max_planes=max_planes, max_topk=8)

    be = backend(args.storage if args.storage != "f32" else "bf16", True, args.serve_slots)
    # warm-up, then capacity: a saturated sample of the job mix (all arriving at once), dispatched in
    # arrival order whatever the policy under test, so that every policy sees the same arrival rate
    calib = serve.Scheduler(be, budget - be.fixed_bytes, args.serve_slots, policy="fifo")
    sample = list(range(min(len(jobs), n_calib)))
    calib.run(requests(None, sample[:6]))
    t0 = time.perf_counter()
    calib.run(requests(None, sample))
    # capacity in evaluations per second (the sample's job mix need not match the stream's), turned
    # into jobs per second with the whole stream's mean work per job
    cap_evals_s = sum(evals[i] for i in sample) / (time.perf_counter() - t0)
    cap_jobs_s = cap_evals_s / (sum(evals.values()) / len(jobs))
    rate = args.serve_load * cap_jobs_s
    served = {}
    for pol in policies:
        sched = serve.Scheduler(be, budget - be.fixed_bytes, args.serve_slots, policy=pol)
        be.intervals_ev.clear()
        with ClockSampler(dev.index) as clk:
            t0 = time.perf_counter()
            done = sched.run(requests(rate))
            wall = time.perf_counter() - t0
        lat = np.array([c.latency for c in done])
        served[pol] = dict(done=done, wall=wall, lat=lat, busy=serve.busy_fraction(be.device_intervals()),
                           peak=sched.peak_bytes + be.fixed_bytes, clocks=clk.summary())
    main = served[policies[-1]]
    done, wall, lat = main["done"], main["wall"], main["lat"]
    del be
    torch.cuda.synchronize(dev)

    # the serial plain-FP32 loop: one job at a time, service time measured per job
    ser = backend("f32", False, 1)
    reqs = requests(rate)
    for r in reqs:
        r.nbytes = ser.estimate(r)
    svc = np.empty(len(reqs))
    for idx, r in enumerate(reqs[:3] + reqs):
        a = time.perf_counter()
        h = ser.admit(r)
        ser.dispatch(h, 0)
        h["done"].synchronize()
        ser.finish(h)
        if idx >= 3:
            svc[idx - 3] = time.perf_counter() - a
    ser_lat = serve.fifo_latencies(np.array([r.arrival for r in reqs]), svc)
    del ser
    ctx.close()
    return dict(policies=policies, jobs=jobs, done=done, wall=wall, lat=lat, main=main, served=served,
                evals=evals, reqs=reqs, svc=svc, ser_lat=ser_lat, rate=rate, cap_jobs_s=cap_jobs_s, t_gen=t_gen)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batch":
        run_batch(args)
    elif args.workload == "serve":
        run_serve(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
