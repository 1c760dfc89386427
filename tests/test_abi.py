"""The C ABI library builds, loads and exports every entry point include/vpgs.h declares.

These tests make no compute call, so they run without a GPU.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vpgs.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(vpgs_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2505_18992_gb300.build import build
    build()
    from paper_2505_18992_gb300 import vpgs
    return vpgs.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header(lib):
    from paper_2505_18992_gb300 import vpgs
    assert sorted(vpgs.exported_names()) == _declared()


def test_struct_layouts_match_the_header(lib, tmp_path):
    """ctypes mirrors against sizeof/offsetof from a C compiler reading the header."""
    import shutil
    import subprocess
    from paper_2505_18992_gb300 import vpgs as C
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = ["vpgs_camera", "vpgs_render_opts", "vpgs_gaussians", "vpgs_gaussian_buffers",
               "vpgs_images", "vpgs_render_stats", "vpgs_anchors", "vpgs_mlp", "vpgs_decode_opts",
               "vpgs_icp_opts", "vpgs_icp_report", "vpgs_icp_map_info", "vpgs_anchor_update_opts",
               "vpgs_spawn_opts"]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vpgs.h"', "int main(void) {"]
    for st in structs:
        lines.append(f'printf("{st} %zu\\n", sizeof({st}));')
        for fname, _ in getattr(C, st)._fields_:
            lines.append(f'printf("{st}.{fname} %zu\\n", offsetof({st}, {fname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.splitlines())
    for st in structs:
        cls = getattr(C, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for fname, _ in cls._fields_:
            assert int(got[f"{st}.{fname}"]) == getattr(cls, fname).offset, (st, fname)


def test_host_side_validation_without_a_gpu(lib):
    from paper_2505_18992_gb300 import vpgs as C
    o = C.default_opts()
    assert (o.tile_w, o.tile_h) == (16, 16)
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7
    cam = C.vpgs_camera(1200, 680, 600.0, 600.0, 600.0, 340.0)
    n1 = C.vpgs_render_workspace_bytes(1000, 1, ctypes.byref(cam), ctypes.byref(o), 10000)
    n2 = C.vpgs_render_workspace_bytes(1000, 1, ctypes.byref(cam), ctypes.byref(o), 20000)
    assert n1 > 0 and n2 > n1
    for bad in (C.default_opts(tile_w=3), C.default_opts(tile_w=32, tile_h=32), C.default_opts(tile_h=7)):
        assert C.vpgs_render_workspace_bytes(1000, 1, ctypes.byref(cam), ctypes.byref(bad), 10) == 0
    assert C.vpgs_render_workspace_bytes(1000, 1, ctypes.byref(cam), ctypes.byref(C.default_opts(tile_w=32, tile_h=16)), 10) > 0
    assert C.vpgs_status_string(7) == b"internal consistency check failed"
    # NULL arguments are rejected before anything touches the device
    assert C.vpgs_render_fwd(None, 0, None, None, None, 1, None, None, None) == 1
    assert C.vpgs_render_bwd(None, 0, None, None, None, 1, None, None, None, None, None, None, None,
                             None) == 1
    assert C.vpgs_pose_step(None, None, None, 1, None, None) == 1
    assert C.vpgs_status_string(2) == b"tile-instance capacity exceeded"
    assert C.vpgs_version().count(b".") == 2
