"""C-ABI boundary checks that need no GPU: exports, struct layout, host-side offsets."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "kb.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1901_02492_gb300 import build
    build.build()
    from paper_1901_02492_gb300 import binding
    return binding


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kb_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    so = ctypes.CDLL(lib.LIB_PATH)
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing
    assert sorted(lib.EXPORTED) == names


def test_result_struct_layout_matches_binding(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "kb.h"\nint main(void){'
                   'printf("%zu", sizeof(kb_result));'
                   + "".join('printf(" %%zu", offsetof(kb_result, %s));' % f for f in
                             ["x0", "y0", "vidx", "nobs", "vx", "vy", "psi", "phi", "nu", "alpha"])
                   + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    from paper_1901_02492_gb300 import binding
    dt = binding.RESULT_DTYPE
    assert vals[0] == dt.itemsize
    assert vals[1:] == [dt.fields[f][1] for f in dt.names]


def test_batch_struct_layouts_match_binding(tmp_path, lib):
    fields = {"kb_batch_item": ["job", "stack", "times", "vx", "vy", "V", "topk", "nu_min", "flags"],
              "kb_batch_group": ["storage", "index_bits", "variant", "kmax", "n_items", "evals", "tuned_ms",
                                 "schedule", "tuned_ms_launch"]}
    body = ""
    for name, fs in fields.items():
        body += 'printf("%%zu", sizeof(%s));' % name
        body += "".join('printf(" %%zu", offsetof(%s, %s));' % (name, f) for f in fs) + 'printf("\\n");'
    src = tmp_path / "blayout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "kb.h"\nint main(void){' + body
                   + "return 0;}\n")
    exe = tmp_path / "blayout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    for line, (name, fs), cls in zip(lines, fields.items(), [lib._BatchItem, lib.BatchGroup]):
        vals = [int(v) for v in line.split()]
        assert vals[0] == ctypes.sizeof(cls), name
        assert vals[1:] == [getattr(cls, f).offset for f in fs], name


def _c_layout(tmp_path, struct, names):
    src = tmp_path / ("%s.c" % struct)
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "kb.h"\nint main(void){'
                   'printf("%%zu", sizeof(%s));' % struct
                   + "".join('printf(" %%zu", offsetof(%s, %s));' % (struct, f) for f in names) + "return 0;}\n")
    exe = tmp_path / struct
    subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    return [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]


@pytest.mark.parametrize("struct,dtype", [("kb_filtered", "FILTERED_DTYPE"), ("kb_moments", "MOMENTS_DTYPE")])
def test_record_layouts_match_binding(tmp_path, lib, struct, dtype):
    dt = getattr(lib, dtype)
    vals = _c_layout(tmp_path, struct, list(dt.names))
    assert vals[0] == dt.itemsize
    assert vals[1:] == [dt.fields[f][1] for f in dt.names]


@pytest.mark.parametrize("struct,cls", [("kb_moment_cuts", "MomentCuts"), ("kb_cluster_params", "ClusterParams")])
def test_parameter_struct_layouts_match_binding(tmp_path, lib, struct, cls):
    c = getattr(lib, cls)
    names = [f[0] for f in c._fields_]
    vals = _c_layout(tmp_path, struct, names)
    assert vals[0] == ctypes.sizeof(c)
    assert vals[1:] == [getattr(c, f).offset for f in names]


def test_offsets_bit_exact_against_oracle(lib):
    rng = np.random.default_rng(5)
    for trial in range(5):
        N = int(rng.integers(1, 40))
        times = rng.uniform(100.0, 100.0 + rng.uniform(0.01, 60.0), N)
        vx = rng.uniform(-4000, 4000, 300)
        vy = rng.uniform(-4000, 4000, 300)
        a = lib.offsets(times, vx, vy)
        b = oracle.offsets(times, vx, vy)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # exact half-way products and the reference epoch
    times = np.array([5.0, 6.0, 5.5, 5.0])
    vx = np.array([1.5, -1.5, 2.5, -2.5, 0.0, 3.0])
    a = lib.offsets(times, vx, -vx)
    b = oracle.offsets(times, vx, -vx)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.all(a[0][:, 0] == 0) and np.all(a[0][:, 3] == 0)


def test_offsets_reject_out_of_range(lib):
    with pytest.raises(lib.KBError):
        lib.offsets(np.array([0.0, 1.0]), np.array([4096.0]), np.array([0.0]))
    with pytest.raises(lib.KBError):
        lib.offsets(np.array([0.0, 64.0]), np.array([1.0]), np.array([0.0]))
    with pytest.raises(lib.KBError):
        lib.offsets(np.array([0.0, np.nan]), np.array([1.0]), np.array([0.0]))
    lib.offsets(np.array([0.0, 63.9]), np.array([4095.9]), np.array([-4095.9]))


def test_static_psi_phi_wrapper_refuses_host_buffers_before_the_call(lib):
    """kb_make_psi_phi_static gets raw pointers and no buffer sizes, so the binding checks
    every buffer first; host tensors and mismatched shapes never reach the library."""
    import torch
    N, H, W, K = 2, 5, 6, 3
    psf = np.full((N, K, K), 1.0 / 9, np.float32)
    sci = torch.zeros((N, H, W))
    var = torch.ones((N, H, W))
    out = torch.zeros((N, H, W, 2))
    with pytest.raises(ValueError):
        lib.make_psi_phi_static(sci, var, None, psf, out)
    with pytest.raises(ValueError):
        lib.make_psi_phi_static(sci[0], var, None, psf, out)          # not [N][H][W]
    with pytest.raises(ValueError):
        lib.make_psi_phi_static(sci, var, None, psf[:, :2, :], out)   # psf not square
    assert torch.all(out == 0)


def test_build_digest_follows_the_sources(tmp_path, lib):
    """build.up_to_date() compares a digest of the sources, not file times."""
    from paper_1901_02492_gb300 import build
    assert build.up_to_date()
    with open(build.STAMP) as f:
        assert f.read().strip() == build.source_digest()


def test_release_build_is_not_a_debug_build(lib):
    """kb_debug_build needs no device: 0 in the release library; the debug build's
    digest differs (its flags add -DKB_DEBUG), so the two never share a stamp."""
    from paper_1901_02492_gb300 import build
    assert lib.debug_build() is False
    assert build.source_digest(debug=True) != build.source_digest()
    assert build.LIB_DEBUG != build.LIB
