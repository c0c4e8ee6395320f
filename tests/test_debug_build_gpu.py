"""The KB_DEBUG build: search kernels with every gather and shared-memory index checked.

The debug library (libkb_debug.so: the same sources with -DKB_DEBUG) is built here,
and a child process loads it through KB_LIBRARY and runs searches that reach every
checked site: FP32 and 16-bit planes, value lists up to 8 and longer (the predicated
remainder), the rescoring's key-list candidate search, the pruned search, a batch,
on images whose widths leave ragged spans and whose trajectories leave the image.
A second child runs the same searches with the release library.  The debug build
must record no out-of-bounds access, and both must give the same result bytes.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import hashlib, json, math, sys
import numpy as np, torch
sys.path.insert(0, ROOT)
import synth
from paper_1901_02492_gb300 import binding as kb

dev = torch.device("cuda:0")
ctx = kb.Context(0)
h = hashlib.sha256()

def planes(st, storage):
    N, H, W = st.sci.shape
    s = kb.Stack(ctx, N, H, W, storage)
    s.make_psi_phi(torch.from_numpy(st.sci).to(dev), torch.from_numpy(st.var).to(dev), None, st.psf)
    return s

cases = [("f32", 8, 0, -math.inf, 0), ("f32", 12, 0, -math.inf, 1), ("bf16", 8, 0, -math.inf, 2),
         ("f16", 12, 0, -math.inf, 3), ("bf16", 8, kb.KB_RESCORE_FP64, -math.inf, 4),
         ("f32", 8, kb.KB_PRUNE, 3.5, 5)]
for storage, k, flags, nu_min, seed in cases:
    st = synth.small_stack(700 + seed, 6, 70, 301, K=5, nan_frac=0.01, n_angles=8, n_speeds=8, s_hi=40.0,
                           n_sources=3, flux=60.0)
    N, H, W = st.sci.shape
    s = planes(st, storage)
    job = kb.Job(ctx, H, W, N, st.vx.size, k, flags & kb.KB_RESCORE_FP64)
    job.search(s, st.times, st.vx, st.vy, k, nu_min, flags)
    h.update(job.results().tobytes())
    job.free()
    s.free()

stacks, jobs, searches = [], [], []
for i, (storage, k) in enumerate([("f32", 4), ("bf16", 8), ("f32", 12)]):
    st = synth.small_stack(720 + i, 5, 40 + 9 * i, 130 + 33 * i, K=5, n_angles=6, n_speeds=6, s_hi=30.0)
    N, H, W = st.sci.shape
    s = planes(st, storage)
    job = kb.Job(ctx, H, W, N, st.vx.size, k, 0)
    stacks.append(s)
    jobs.append(job)
    searches.append(dict(job=job, stack=s, times=st.times, vx=st.vx, vy=st.vy, topk=k, flags=0))
b = kb.Batch(ctx, searches, autotune=False)
b.run()
for j in jobs:
    h.update(j.results().tobytes())
b.free()
for o in jobs + stacks:
    o.free()
torch.cuda.synchronize()
word = ctx.debug_word() if kb.debug_build() else None
print(json.dumps({"debug": kb.debug_build(), "word": word, "digest": h.hexdigest()}))
ctx.close()
"""


def _child(lib):
    env = dict(os.environ)
    if lib:
        env["KB_LIBRARY"] = lib
    else:
        env.pop("KB_LIBRARY", None)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], capture_output=True, text=True,
                       env=env, cwd=ROOT, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_debug_build_records_nothing_and_matches_release():
    from paper_1901_02492_gb300 import build
    lib = build.build(debug=True)
    dbg = _child(lib)
    rel = _child(None)
    assert dbg["debug"] is True and rel["debug"] is False
    assert dbg["word"] == 0, "out-of-bounds access: site %d, offset %d" % (dbg["word"] >> 56,
                                                                           dbg["word"] & ((1 << 56) - 1))
    assert dbg["digest"] == rel["digest"]
