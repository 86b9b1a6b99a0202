"""FP64 CPU oracle (test infrastructure only).

A plain, slow C++ restatement of what the splat rasterizer computes, used to
check the CUDA path.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the CUDA library and never takes an input from it.

Functions mirror ``oracle.cpp``: projection (Sec. 2.1.1-2.1.2), depth order,
forward compositing with the 1/255 and T-culling rules (Eq. 2, Procedure 1),
and the analytic backward with Eq. 3 / Eq. 4 written as explicit suffix sums.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Tie bands (see trace_pixel in oracle.cpp).  Defaults suit images up to ~2k px.
DEFAULT_BANDS = dict(band_cut=2e-3, band_depth=5e-7, band_t=1e-4, band_near=1e-5, band_clamp=1e-5)


def build(force: bool = False) -> str:
    """Compile liboracle.so (g++, FP64, OpenMP) if missing or older than its source."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB)
    return _lib


def _d(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def camera_array(cam) -> np.ndarray:
    return cam.as_f64_array()


def opts_array(t_cull: float = 1e-4, clamp01: bool = False, quant: int = 0,
               per_fragment: bool = False, **bands) -> np.ndarray:
    b = dict(DEFAULT_BANDS)
    b.update(bands)
    return np.array([t_cull, float(clamp01), float(quant), float(per_fragment), b["band_cut"],
                     b["band_depth"], b["band_t"], b["band_near"], b["band_clamp"]],
                    dtype=np.float64)


QUANT = {"fp32": 0, "fp16": 1, "unorm16": 2, "unorm8": 3}


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(n: int) -> int:
    """Threads the oracle's parallel loops use (0: all cores); returns the count."""
    return int(_load().oracle_set_threads(ctypes.c_int(int(n))))


def sh_basis(deg: int, dirs: np.ndarray, grad: bool = False):
    dirs = _d(dirs).reshape(-1, 3)
    n = dirs.shape[0]
    K = (deg + 1) ** 2
    Y = np.zeros((n, K))
    dY = np.zeros((n, K, 3)) if grad else None
    rc = _load().oracle_sh_basis(ctypes.c_int(deg), _ptr(dirs), ctypes.c_int(n), _ptr(Y), _ptr(dY))
    assert rc == 0
    return (Y, dY) if grad else Y


def _scene_args(scene):
    m, s, q, o, sh = (_d(a) for a in scene.arrays())
    return (m, s, q, o, sh), [ctypes.c_int(scene.n), _ptr(m), _ptr(s), _ptr(q), _ptr(o), _ptr(sh),
                              ctypes.c_int(scene.sh_degree)]


def project(scene, cam, clamp01: bool = False) -> np.ndarray:
    """[N, 20]: valid, mu2(2), Sigma2D(00,01,11), conic(a,b,c), rgb(3), depth,
    raw rgb(3), camera-space t(3), unused."""
    keep, args = _scene_args(scene)
    camv = camera_array(cam)
    out = np.zeros((scene.n, 20))
    rc = _load().oracle_project(*args, _ptr(camv), ctypes.c_int(int(clamp01)), _ptr(out))
    assert rc == 0
    return out


def stable_sort_u32(keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, dtype=np.uint32)
    order = np.zeros(keys.shape[0], dtype=np.int32)
    _load().oracle_stable_sort_u32(ctypes.c_int(keys.shape[0]), _ptr(keys), _ptr(order))
    return order


def depth_order(scene, cam) -> np.ndarray:
    keep, args = _scene_args(scene)
    camv = camera_array(cam)
    order = np.zeros(scene.n, dtype=np.int32)
    n = _load().oracle_depth_order(*args, _ptr(camv), _ptr(order))
    return order[:n]


def render(scene, cam, opts=None, pixels=None, timings: bool = False):
    """Forward render.  Returns dict(color [P,3] or [H,W,3], T, nfrag, last, ambig)
    (and timings: seconds of preprocessing and of tracing)."""
    opts = opts_array() if opts is None else opts
    keep, args = _scene_args(scene)
    camv = camera_array(cam)
    if pixels is None:
        npix = cam.width * cam.height
        pix = None
    else:
        pix = np.ascontiguousarray(pixels, dtype=np.int32)
        npix = pix.shape[0]
    color = np.zeros((npix, 3))
    T = np.zeros(npix)
    nfrag = np.zeros(npix, dtype=np.int32)
    last = np.zeros(npix, dtype=np.int32)
    ambig = np.zeros(npix, dtype=np.int32)
    tm = np.zeros(2)
    rc = _load().oracle_render(*args, _ptr(camv), _ptr(opts), _ptr(pix), ctypes.c_int(npix),
                               _ptr(color), _ptr(T), _ptr(nfrag), _ptr(last), _ptr(ambig),
                               _ptr(tm))
    assert rc == 0
    out = dict(color=color, T=T, nfrag=nfrag, last=last, ambig=ambig)
    if pixels is None:
        H, W = cam.height, cam.width
        out = {k: v.reshape((H, W, 3) if k == "color" else (H, W)) for k, v in out.items()}
    if timings:
        out["timings"] = dict(preprocess_s=float(tm[0]), trace_s=float(tm[1]))
    return out


def backward(scene, cam, dLdC, opts=None, quant_cprime: bool = False, pixels=None,
             timings: bool = False):
    """Analytic backward for dL/dC [H, W, 3].  Returns dict of gradients
    (means, scales, quats, opacities, sh), the per-splat 2D gradients g2d [N, 9]
    (mu2 x/y, conic a/b/c, rgb, opacity) and the image.  With `pixels`, only
    those pixels (linear index y*W+x) are traced and contribute."""
    opts = opts_array() if opts is None else opts
    keep, args = _scene_args(scene)
    camv = camera_array(cam)
    g = _d(dLdC).reshape(cam.height, cam.width, 3)
    N, K = scene.n, (scene.sh_degree + 1) ** 2
    image = np.zeros((cam.height, cam.width, 3))
    gm, gs, gq, go = np.zeros((N, 3)), np.zeros((N, 3)), np.zeros((N, 4)), np.zeros(N)
    gsh = np.zeros((N, K, 3))
    g2d = np.zeros((N, 9))
    pix = None if pixels is None else np.ascontiguousarray(pixels, dtype=np.int32)
    tm = np.zeros(2)
    rc = _load().oracle_backward(*args, _ptr(camv), _ptr(opts), _ptr(g), ctypes.c_int(int(quant_cprime)),
                                 _ptr(pix), ctypes.c_int(0 if pix is None else pix.shape[0]),
                                 _ptr(image), _ptr(gm), _ptr(gs), _ptr(gq), _ptr(go), _ptr(gsh),
                                 _ptr(g2d), _ptr(tm))
    assert rc == 0
    out = dict(means=gm, scales=gs, quats=gq, opacities=go, sh=gsh, g2d=g2d, image=image)
    if timings:
        out["timings"] = dict(preprocess_s=float(tm[0]), trace_s=float(tm[1]))
    return out


def splat_grads(scene, cam, dLdC, ids, opts=None):
    """Gradients of selected splats only (tracing just their footprint pixels)."""
    opts = opts_array() if opts is None else opts
    keep, args = _scene_args(scene)
    camv = camera_array(cam)
    g = _d(dLdC).reshape(cam.height, cam.width, 3)
    ids = np.ascontiguousarray(ids, dtype=np.int32)
    n, K = ids.shape[0], (scene.sh_degree + 1) ** 2
    g2d = np.zeros((n, 9))
    gm, gs, gq, go = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros((n, 4)), np.zeros(n)
    gsh = np.zeros((n, K, 3))
    cnt = np.zeros(n, dtype=np.int32)
    rc = _load().oracle_splat_grads(*args, _ptr(camv), _ptr(opts), _ptr(g), _ptr(ids), ctypes.c_int(n),
                                    _ptr(g2d), _ptr(gm), _ptr(gs), _ptr(gq), _ptr(go), _ptr(gsh),
                                    _ptr(cnt))
    assert rc == 0
    return dict(means=gm, scales=gs, quats=gq, opacities=go, sh=gsh, g2d=g2d, pixels=cnt)
