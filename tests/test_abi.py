"""The C ABI library loads and exports every entry point include/gsr.h
declares; the ctypes structs match the header's layout.  CPU only."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsr.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2505_18764_gb300 import build
    build.build_library()
    from paper_2505_18764_gb300 import _lib
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), f"{n} declared in gsr.h but not exported"
    from paper_2505_18764_gb300 import _lib
    assert set(names) == set(_lib.EXPORTED)


def test_struct_layout_matches_header(tmp_path):
    from paper_2505_18764_gb300 import _lib
    src = tmp_path / "layout.c"
    checks = {
        "gs_camera": (_lib.GsCamera, ["viewmat", "campos", "fx", "width", "height", "znear"]),
        "gs_raster_opts": (_lib.GsRasterOpts, ["state_format", "t_cull", "pair_capacity"]),
        "gs_workspace": (_lib.GsWorkspace, ["base", "bytes", "pair_cap", "n", "pair_passes", "layout"]),
        "gs_scene_ref": (_lib.GsSceneRef, ["means", "sh", "n", "sh_degree"]),
        "gs_request": (_lib.GsRequest, ["scene", "camera", "opts", "mode", "loss_kind", "image",
                                         "loss", "d_sh"]),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void){"]
    for cname, (_, fields) in checks.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in fields:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for line in out:
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    for cname, (cls, fields) in checks.items():
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for f in fields:
            assert got[(cname, f)] == getattr(cls, f).offset, f"{cname}.{f}"


def test_workspace_size_and_argument_errors(lib):
    from paper_2505_18764_gb300 import _lib, RasterOpts
    o = RasterOpts().to_c()
    n = ctypes.c_size_t(0)
    assert lib.gs_workspace_size(1000, 128, 128, ctypes.byref(o), ctypes.byref(n)) == 0
    assert n.value > 1000 * 48 * 3
    # bad options are rejected on the host, with a message
    o.state_format = 9
    assert lib.gs_workspace_size(1000, 128, 128, ctypes.byref(o), ctypes.byref(n)) == _lib.GS_ERR_INVALID_ARG
    assert b"state_format" in lib.gs_last_error()
    o = RasterOpts().to_c()
    assert lib.gs_workspace_size(-1, 128, 128, ctypes.byref(o), ctypes.byref(n)) == _lib.GS_ERR_INVALID_ARG
    ws = _lib.GsWorkspace()
    # a null device pointer is refused before any CUDA call
    assert lib.gs_workspace_init(ctypes.byref(ws), None, 1 << 20, 10, 16, 16, ctypes.byref(o), None) == _lib.GS_ERR_INVALID_ARG
    # calls on an uninitialised workspace are refused before any CUDA call
    assert lib.gs_sort(ctypes.byref(_lib.GsWorkspace()), None) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_loss(None, None, 10, 7, None, None, None) == _lib.GS_ERR_INVALID_ARG
    blank = ctypes.byref(_lib.GsWorkspace())
    assert lib.gs_zero_touched_gradients(blank, 0, None, None, None, None, None, None) == \
        _lib.GS_ERR_INVALID_ARG
    assert b"workspace" in lib.gs_last_error()
    # the graph form of the batch call validates like the direct one, before any capture
    assert lib.gs_render_batch_graph(None, 1, blank, None) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_render_batch_graph(None, -1, blank, None) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_render_batch_graph(None, 0, blank, None) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_graph_release(blank) == _lib.GS_OK   # nothing kept: a no-op


def test_package_fails_loudly_without_library(tmp_path):
    from paper_2505_18764_gb300 import _lib
    with pytest.raises(RuntimeError, match="not built"):
        _lib.load.__wrapped__(str(tmp_path / "missing.so")) if hasattr(_lib.load, "__wrapped__") else \
            _load_missing(_lib, str(tmp_path / "missing.so"))


def _load_missing(_lib, path):
    saved = _lib._lib
    _lib._lib = None
    try:
        _lib.load(path)
    finally:
        _lib._lib = saved
