"""In-tree build of libkb.so (the C-ABI library with the sm_103a kernels).

Each translation unit under csrc/ is compiled by nvcc in parallel for
sm_103a only, then linked into paper_1901_02492_gb300/libkb.so next to this
file.  No cmake, no torch extension machinery.  build(debug=True) makes
libkb_debug.so instead: the same sources with -DKB_DEBUG, whose search kernels
check every gather and shared-memory index and record the first one out of
bounds (kb_debug_word) instead of making it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libkb.so")
STAMP = LIB + ".sha256"     # digest of the sources and flags the library was built from
LIB_DEBUG = os.path.join(HERE, "libkb_debug.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

NVCC = os.environ.get("NVCC", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fno-strict-aliasing",
         "-I", INCLUDE]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.h")) + [os.path.join(INCLUDE, "kb.h"), __file__]


def _flags(debug: bool):
    return FLAGS + (["-DKB_DEBUG"] if debug else [])


def source_digest(debug: bool = False) -> str:
    """sha256 over every input of the build (sources, headers, this script) and the
    compiler flags.  File times are not used: a copied tree keeps the times of the
    copy, so a library newer than changed sources would otherwise be reused."""
    h = hashlib.sha256()
    h.update(" ".join([NVCC] + ARCH + _flags(debug)).encode())
    for d in sorted(set(_deps())):
        h.update(os.path.relpath(d, os.path.dirname(HERE)).encode())
        with open(d, "rb") as f:
            h.update(hashlib.sha256(f.read()).digest())
    return h.hexdigest()


def up_to_date(debug: bool = False) -> bool:
    lib = LIB_DEBUG if debug else LIB
    stamp = lib + ".sha256"
    if not (os.path.exists(lib) and os.path.exists(stamp)):
        return False
    with open(stamp) as f:
        return f.read().strip() == source_digest(debug)


def build(force: bool = False, verbose: bool = False, debug: bool = False) -> str:
    """Compile and link libkb.so (libkb_debug.so with debug=True); returns its path."""
    lib = LIB_DEBUG if debug else LIB
    stamp = lib + ".sha256"
    if not force and up_to_date(debug):
        return lib
    digest = source_digest(debug)
    bdir = BUILD + ("_debug" if debug else "")
    os.makedirs(bdir, exist_ok=True)
    srcs = _sources()
    flags = _flags(debug)

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        cmd = [NVCC] + ARCH + flags + ["-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        results = list(ex.map(compile_one, srcs))
    if verbose:
        for _, log in results:
            print(log)
    objs = [o for o, _ in results]
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    with open(stamp + ".tmp%d" % os.getpid(), "w") as f:
        f.write(digest + "\n")
    os.replace(stamp + ".tmp%d" % os.getpid(), stamp)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
