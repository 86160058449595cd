"""The C-ABI library loads, exports every function include/*.h declares, the
binding's ctypes structures have the header's layout, and
rejects bad arguments on the host (no GPU needed for any of this)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2310_10642_gb300 import inputs as I
from paper_2310_10642_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    N.build()
    return N.lib()


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//.*", "", text)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(fgs4d_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_the_path():
    names = declared_functions()
    for fn in ("fgs4d_slice_project", "fgs4d_bin_sort", "fgs4d_render", "fgs4d_render_backward"):
        assert fn in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for fn in names:
        assert hasattr(lib, fn), f"{fn} declared but not exported"
    assert set(N.EXPORTS) <= set(names)


def test_version_and_status_strings(lib):
    assert lib.fgs4d_abi_version() == 5
    for code in range(6):
        assert len(lib.fgs4d_status_string(code)) > 0


def test_default_options_match_readings(lib):
    o = N.fgs4d_default_options()
    assert abs(o.p_min - 0.05) < 1e-7 and abs(o.near_z - 0.2) < 1e-7
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7
    assert abs(o.T_min - 1e-4) < 1e-10 and abs(o.dilation - 0.3) < 1e-7
    assert o.tile_size == 16 and o.batch_depth == 256 and o.record_fp16 == 0 and o.bin_size == 0


def _views(k=2, w=100, h=60):
    return N.make_views([I.view((0, 0, 4), w, h, 0.5) for _ in range(k)])


def test_state_size_grows_with_capacity(lib):
    o = N.fgs4d_default_options()
    v = _views()
    a = N.fgs4d_state_size(1000, v, 2, 0, o)
    b = N.fgs4d_state_size(1000, v, 2, 100000, o)
    assert 4 * 100000 <= b - a < 4 * 100000 + 1024  # counting path: one array of splat ids
    # a view of more than 4096 binning tiles takes the radix path (keys and values, double-buffered)
    big = N.make_views([I.view((0, 0, 4), 1600, 1400, 0.5)])  # 100 x 88 tiles of 16 pixels
    assert N.fgs4d_state_size(1000, big, 1, 100000, o) - N.fgs4d_state_size(1000, big, 1, 0, o) >= 16 * 100000
    info = N.fgs4d_state_layout(1000, v, 2, o, b)
    assert 100000 <= info.pair_capacity < 100000 + 64 and info.n_splats == 2000
    assert info.total_tiles == 2 * 7 * 4
    # binning tiles of 64 pixels: 2 x 1 per 100 x 60 view
    o64 = N.make_options(dict(tile_size=32, bin_size=64))
    assert N.fgs4d_state_layout(1000, v, 2, o64, N.fgs4d_state_size(1000, v, 2, 100, o64)).total_tiles == 2 * 2 * 1
    assert N.fgs4d_total_pixels(v, 2) == 2 * 6000


def test_invalid_arguments_rejected_on_host(lib):
    o = N.fgs4d_default_options()
    v = _views()
    size = ctypes.c_size_t()
    # bad view count, negative n, bad capacity
    assert lib.fgs4d_state_size(10, v, 0, 10, ctypes.byref(o), ctypes.byref(size)) == 1
    assert lib.fgs4d_state_size(10, v, N.MAX_VIEWS + 1, 10, ctypes.byref(o), ctypes.byref(size)) == 1
    assert lib.fgs4d_state_size(-1, v, 2, 10, ctypes.byref(o), ctypes.byref(size)) == 1
    assert lib.fgs4d_state_size(10, v, 2, -5, ctypes.byref(o), ctypes.byref(size)) == 1
    # bad options
    for field, val in (("alpha_max", 1.5), ("alpha_min", 0.0), ("near_z", 0.0), ("T_min", float("nan")),
                       ("tile_size", 8), ("batch_depth", 100), ("batch_depth", 512), ("record_fp16", 2),
                       ("bin_size", 8), ("bin_size", 48), ("bin_size", 128), ("bin_size", -16),
                       ("accumulate_grads", 2), ("accumulate_grads", -1)):
        bad = N.fgs4d_default_options()
        setattr(bad, field, val)
        assert lib.fgs4d_state_size(10, v, 2, 10, ctypes.byref(bad), ctypes.byref(size)) == 1
    # a binning tile smaller than the compositing tile
    bad = N.make_options(dict(tile_size=32, bin_size=16))
    assert lib.fgs4d_state_size(10, v, 2, 10, ctypes.byref(bad), ctypes.byref(size)) == 1
    # bad view sizes
    bv = _views(1, 0, 10)
    assert lib.fgs4d_state_size(10, bv, 1, 10, ctypes.byref(o), ctypes.byref(size)) == 1
    # null / misaligned state and null gaussian arrays are rejected before any launch
    g = N.Gaussians(None, None, None, None, None, None, 10, 1, 1, 1.0, 0)
    assert lib.fgs4d_slice_project(ctypes.byref(g), v, 2, ctypes.byref(o), None, 0, None) == 1
    g2 = N.Gaussians(16, 32, 48, 64, 80, 96, 10, 5, 1, 1.0, 0)  # sh degree out of range
    assert lib.fgs4d_slice_project(ctypes.byref(g2), v, 2, ctypes.byref(o), 256, 1 << 20, None) == 1
    g3 = N.Gaussians(16, 32, 48, 64, 80, 96, 10, 1, 1, 0.0, 0)  # period 0
    assert lib.fgs4d_slice_project(ctypes.byref(g3), v, 2, ctypes.byref(o), 256, 1 << 20, None) == 1
    g5 = N.Gaussians(16, 32, 48, 64, 80, 96, 10, 1, 1, 1.0, 0, 7)  # unknown rotation mode
    assert lib.fgs4d_slice_project(ctypes.byref(g5), v, 2, ctypes.byref(o), 256, 1 << 20, None) == 1
    g6 = N.Gaussians(16, 32, 48, None, 80, 96, 10, 1, 1, 1.0, 0, N.ROT_4D)  # 4D rotation needs q_right
    assert lib.fgs4d_slice_project(ctypes.byref(g6), v, 2, ctypes.byref(o), 256, 1 << 20, None) == 1
    g7 = N.Gaussians(16, 32, 48, None, 80, 96, 10, 1, 1, 1.0, 0, N.ROT_STATIC + 1)  # one past the last mode
    assert lib.fgs4d_slice_project(ctypes.byref(g7), v, 2, ctypes.byref(o), 256, 1 << 20, None) == 1
    g4 = N.Gaussians(16, 32, 48, 64, 80, 97, 10, 1, 1, 1.0, 0)  # misaligned shs
    assert lib.fgs4d_slice_project(ctypes.byref(g4), v, 2, ctypes.byref(o), 256, 1 << 20, None) == 1
    # state smaller than the fixed part
    assert lib.fgs4d_bin_sort(10, v, 2, ctypes.byref(o), 256, 1024, None) == 2
    assert lib.fgs4d_render(10, v, 2, ctypes.byref(o), 256, 1 << 30, None, None, None, None) == 1
    # work counters: null and misaligned stats are rejected
    assert lib.fgs4d_render_stats(10, v, 2, ctypes.byref(o), 256, 1 << 30, 256, 512, 768, None, None) == 1
    assert lib.fgs4d_render_stats(10, v, 2, ctypes.byref(o), 256, 1 << 30, 256, 512, 768, 1028, None) == 1


# ctypes mirror of each header struct: (binding class, C type name)
STRUCTS = [("Gaussians", "fgs4d_gaussians"), ("View", "fgs4d_view"), ("Options", "fgs4d_options"),
           ("GaussianGrads", "fgs4d_gaussian_grads"), ("Counters", "fgs4d_counters"),
           ("AdamGroup", "fgs4d_adam_group"), ("StateLayoutInfo", "fgs4d_state_layout_info")]


# binding constants mirroring the header's: (name in native.py, C expression)
CONSTANTS = [("MAX_VIEWS", "FGS4D_MAX_VIEWS"), ("TILE", "FGS4D_TILE"), ("F32", "FGS4D_F32"), ("BF16", "FGS4D_BF16"),
             ("ROT_4D", "FGS4D_ROT_4D"), ("ROT_SPATIAL", "FGS4D_ROT_SPATIAL"), ("ROT_STATIC", "FGS4D_ROT_STATIC"),
             ("STATUS_PAIR_OVERFLOW", "FGS4D_STATUS_PAIR_OVERFLOW"), ("STATUS_NONFINITE", "FGS4D_STATUS_NONFINITE"),
             ("NOALLOC_MAX_SPLATS", "FGS4D_NOALLOC_MAX_SPLATS")]


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes structure of the binding has the size, field names and
    field offsets that a C compiler gives the header's struct, and the
    binding's constants the header's values (compiled here with the host
    gcc; the header is plain C)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "fgs4d.h"', "int main(void) {"]
    for cls, ctype in STRUCTS:
        lines.append(f'  printf("{cls} size %zu\\n", sizeof({ctype}));')
        for name, _ in getattr(N, cls)._fields_:
            lines.append(f'  printf("{cls} {name} %zu\\n", offsetof({ctype}, {name}));')
    for py, c in CONSTANTS:
        lines.append(f'  printf("const {py} %lld\\n", (long long)({c}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cls, name, val = line.split()
        got[(cls, name)] = int(val)
    for py, c in CONSTANTS:
        assert getattr(N, py) == got[("const", py)], (py, c)
    for cls, ctype in STRUCTS:
        s = getattr(N, cls)
        assert ctypes.sizeof(s) == got[(cls, "size")], (cls, ctypes.sizeof(s), got[(cls, "size")])
        for name, _ in s._fields_:
            assert getattr(s, name).offset == got[(cls, name)], (cls, name)
