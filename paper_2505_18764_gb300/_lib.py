"""ctypes view of libgsr.so: the structs and function signatures of include/gsr.h.

Argument marshalling only.  Loading fails loudly when the CUDA library has
not been built; there is no other implementation to fall back to.
"""
from __future__ import annotations

import ctypes
import os
import threading

from ctypes import (POINTER, Structure, c_double, c_float, c_int32, c_int64, c_size_t, c_uint32,
                    c_uint64, c_void_p, c_char_p)

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgsr.so")

GS_OK = 0
GS_ERR_INVALID_ARG = -1
GS_ERR_CAPACITY = -2
GS_ERR_TIMEOUT = -3
GS_ERR_CUDA = -4

GS_STATE_FP32, GS_STATE_FP16, GS_STATE_UNORM16, GS_STATE_UNORM8 = 0, 1, 2, 3
GS_REDUCE_WARP, GS_REDUCE_NAIVE, GS_REDUCE_FRAGMENT = 0, 1, 2
GS_SPLIT_THRESHOLD_DEFAULT = 1536
GS_REDUCE_THRESHOLD_DEFAULT = 16
GS_BWD_FRONT_TO_BACK, GS_BWD_BACK_TO_FRONT = 0, 1
GS_MODE_FORWARD, GS_MODE_FORWARD_BACKWARD = 0, 1
GS_LOSS_NONE, GS_LOSS_L1, GS_LOSS_L2 = 0, 1, 2
GS_SORT_NOALLOC_MAX_PAIRS = 262144
(GS_ARRAY_SORTED_IDS, GS_ARRAY_DEPTH_KEYS, GS_ARRAY_RECORDS, GS_ARRAY_PAIR_BLOCKS,
 GS_ARRAY_PAIR_RANKS, GS_ARRAY_RANGES, GS_ARRAY_GRAD2D, GS_ARRAY_BOXES) = range(8)


class GsCamera(Structure):
    _fields_ = [("viewmat", c_float * 12), ("campos", c_float * 3), ("fx", c_float),
                ("fy", c_float), ("cx", c_float), ("cy", c_float), ("width", c_int32),
                ("height", c_int32), ("znear", c_float)]


class GsRasterOpts(Structure):
    _fields_ = [("state_format", c_int32), ("reduce_mode", c_int32),
                ("reduce_threshold", c_int32), ("sh_degree", c_int32), ("t_cull", c_float),
                ("split_threshold", c_int32), ("backward_order", c_int32), ("chunked", c_int32),
                ("pair_capacity", c_int64)]


class GsWorkspace(Structure):
    _fields_ = [("base", c_void_p), ("bytes", c_size_t), ("n_cap", c_int32),
                ("width_cap", c_int32), ("height_cap", c_int32), ("chunked", c_int32),
                ("pair_cap", c_int64), ("n", c_int32), ("width", c_int32), ("height", c_int32),
                ("sh_degree", c_int32), ("state_format", c_int32), ("clamp01", c_int32),
                ("pair_passes", c_int32), ("n_chunks", c_int32), ("layout", c_uint64 * 24)]


class GsSceneRef(Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p),
                ("opacities", c_void_p), ("sh", c_void_p), ("n", c_int32), ("sh_degree", c_int32)]


class GsRequest(Structure):
    _fields_ = [("scene", GsSceneRef), ("camera", GsCamera), ("opts", GsRasterOpts),
                ("mode", c_int32), ("loss_kind", c_int32), ("image", c_void_p),
                ("state", c_void_p), ("last", c_void_p), ("n_contrib", c_void_p),
                ("target", c_void_p), ("dL_dimage", c_void_p), ("loss", c_void_p),
                ("d_means", c_void_p), ("d_scales", c_void_p), ("d_quats", c_void_p),
                ("d_opacities", c_void_p), ("d_sh", c_void_p), ("zero_touched", c_int32),
                ("pad0", c_int32), ("loss_host", c_void_p)]


_SIGS = {
    "gs_workspace_size": [c_int32, c_int32, c_int32, POINTER(GsRasterOpts), POINTER(c_size_t)],
    "gs_workspace_init": [POINTER(GsWorkspace), c_void_p, c_size_t, c_int32, c_int32, c_int32,
                          POINTER(GsRasterOpts), c_void_p],
    "gs_project": [POINTER(GsWorkspace), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                   c_int32, POINTER(GsCamera), POINTER(GsRasterOpts), c_void_p],
    "gs_sort": [POINTER(GsWorkspace), c_void_p],
    "gs_raster_forward": [POINTER(GsWorkspace), POINTER(GsCamera), POINTER(GsRasterOpts),
                          c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
    "gs_raster_backward": [POINTER(GsWorkspace), c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                           c_int32, POINTER(GsCamera), POINTER(GsRasterOpts), c_void_p, c_void_p,
                           c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
    "gs_bin": [POINTER(GsWorkspace), POINTER(GsCamera), POINTER(GsRasterOpts), c_void_p],
    "gs_blend_forward": [POINTER(GsWorkspace), POINTER(GsCamera), POINTER(GsRasterOpts),
                         c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
    "gs_blend_backward": [POINTER(GsWorkspace), POINTER(GsCamera), POINTER(GsRasterOpts),
                          c_void_p, c_void_p, c_void_p, c_void_p],
    "gs_project_backward": [POINTER(GsWorkspace), c_void_p, c_void_p, c_void_p, c_void_p,
                            c_void_p, c_int32, POINTER(GsCamera), POINTER(GsRasterOpts),
                            c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
    "gs_loss": [c_void_p, c_void_p, c_int64, c_int32, c_void_p, c_void_p, c_void_p],
    "gs_render_batch": [POINTER(GsRequest), c_int32, POINTER(GsWorkspace), c_void_p],
    "gs_render_batch_graph": [POINTER(GsRequest), c_int32, POINTER(GsWorkspace), c_void_p],
    "gs_graph_release": [POINTER(GsWorkspace)],
    "gs_check_status": [POINTER(GsWorkspace), c_void_p],
    "gs_workspace_sort_bytes": [POINTER(GsWorkspace), POINTER(c_size_t), POINTER(c_size_t)],
    "gs_read_counters": [POINTER(GsWorkspace), POINTER(c_int64), c_void_p],
    "gs_copy_array": [POINTER(GsWorkspace), c_int32, c_void_p, c_size_t, c_void_p],
    "gs_sort_pairs": [POINTER(GsWorkspace), c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                      c_int32, c_void_p],
    "gs_sort_pairs_noalloc": [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_int32, c_void_p],
    "gs_sort_pairs_noalloc_status": [c_void_p],
    "gs_test_stalled_sort": [POINTER(GsWorkspace), c_void_p, c_void_p, c_void_p, c_void_p, c_int32,
                             c_uint32, c_void_p],
    "gs_fp32_fma_rate": [c_int32, POINTER(c_double), c_void_p],
    "gs_raster_forward_slab": [POINTER(GsWorkspace), POINTER(GsCamera), POINTER(GsRasterOpts),
                               c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p],
    "gs_raster_backward_slab": [POINTER(GsWorkspace), c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_int32, POINTER(GsCamera), POINTER(GsRasterOpts),
                                c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                c_void_p],
    "gs_slab_composite": [c_void_p, c_int32, c_int32, c_int64, c_void_p, c_void_p, c_void_p,
                          c_void_p, c_void_p],
    "gs_zero_touched_gradients": [POINTER(GsWorkspace), c_int32, c_void_p, c_void_p, c_void_p,
                                  c_void_p, c_void_p, c_void_p],
}

EXPORTED = tuple(_SIGS) + ("gs_last_error",)

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Loads libgsr.so.  Raises if it is missing: build it with
    ``python -m paper_2505_18764_gb300.build`` (or __graft_entry__.build())."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} is missing "
                                   "(run paper_2505_18764_gb300/build.py)")
            lib = ctypes.CDLL(path)
            for name, args in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = c_int32
            lib.gs_last_error.argtypes = []
            lib.gs_last_error.restype = c_char_p
            _lib = lib
    return _lib


class GsError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with {code}: {msg}")
        self.code = code


def check(code: int, where: str):
    if code != GS_OK:
        msg = load().gs_last_error().decode(errors="replace")
        raise GsError(code, where, msg)
