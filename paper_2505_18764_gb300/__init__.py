"""GB300 differentiable Gaussian-splat rasterizer (arXiv 2505.18764, Sec. 3).

Thin Python layer over the C ABI in include/gsr.h: PyTorch supplies device
memory and streams; every step of the forward and backward pass runs in the
CUDA kernels of libgsr.so.  Function names follow the C entry points.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import torch

from . import _lib
from ._lib import (GS_LOSS_L1, GS_LOSS_L2, GS_LOSS_NONE, GS_MODE_FORWARD, GS_MODE_FORWARD_BACKWARD,
                   GsError, check)

STATE_FORMATS = {"fp32": 0, "fp16": 1, "unorm16": 2, "unorm8": 3}
STATE_BYTES = {"fp32": 16, "fp16": 8, "unorm16": 8, "unorm8": 4}
REDUCE_MODES = {"warp": 0, "naive": 1, "fragment": 2}
BACKWARD_ORDERS = {"front_to_back": 0, "back_to_front": 1}
NONE_RANK = 0xFFFFFFFF


@dataclass
class RasterOpts:
    """Mirror of gs_raster_opts."""
    state_format: str = "fp32"
    reduce_mode: str = "warp"
    reduce_threshold: int = 0
    sh_degree: int = 0
    t_cull: float = 1e-4
    pair_capacity: int = 0
    split_threshold: int = 0
    backward_order: str = "front_to_back"
    chunked: bool = False

    def to_c(self) -> _lib.GsRasterOpts:
        o = _lib.GsRasterOpts()
        o.state_format = STATE_FORMATS[self.state_format]
        o.reduce_mode = REDUCE_MODES[self.reduce_mode]
        o.reduce_threshold = int(self.reduce_threshold)
        o.sh_degree = int(self.sh_degree)
        o.t_cull = float(self.t_cull)
        o.pair_capacity = int(self.pair_capacity)
        o.split_threshold = int(self.split_threshold)
        o.backward_order = BACKWARD_ORDERS[self.backward_order]
        o.chunked = int(bool(self.chunked))
        return o


def camera_to_c(cam) -> _lib.GsCamera:
    """Any object with viewmat [3,4], campos [3], fx, fy, cx, cy, width, height, znear
    (a GsCamera passes through unchanged)."""
    if isinstance(cam, _lib.GsCamera):
        return cam
    c = _lib.GsCamera()
    vm = [float(v) for v in torch.as_tensor(cam.viewmat, dtype=torch.float32).reshape(-1).tolist()]
    for i in range(12):
        c.viewmat[i] = vm[i]
    cp = [float(v) for v in torch.as_tensor(cam.campos, dtype=torch.float32).reshape(-1).tolist()]
    for i in range(3):
        c.campos[i] = cp[i]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.znear = float(getattr(cam, "znear", 0.2))
    return c


@dataclass
class SceneTensors:
    """Device-resident splat parameters (activated values, float32, contiguous)."""
    means: torch.Tensor
    scales: torch.Tensor
    quats: torch.Tensor
    opacities: torch.Tensor
    sh: torch.Tensor
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @staticmethod
    def from_numpy(scene, device="cuda") -> "SceneTensors":
        def t(a):
            return torch.as_tensor(a, dtype=torch.float32).contiguous().to(device)
        return SceneTensors(t(scene.means), t(scene.scales), t(scene.quats), t(scene.opacities),
                            t(scene.sh), int(scene.sh_degree))

    def tensors(self):
        return self.means, self.scales, self.quats, self.opacities, self.sh


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


def _ptr(t, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _f32(t, name):
    if t is not None and t.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    return _ptr(t, name)


def _need(t, numel, name, min_bytes_per=None):
    """The C ABI cannot see tensor sizes: refuse any buffer smaller than the call will touch."""
    if t is None:
        return
    if t.numel() * t.element_size() < numel * (min_bytes_per or t.element_size()):
        raise ValueError(f"{name} holds {t.numel()} elements, the call needs {numel}")


def _check_scene(scene: "SceneTensors", sh_degree: int):
    n = scene.n
    K = (sh_degree + 1) ** 2
    if tuple(scene.means.shape) != (n, 3) or tuple(scene.scales.shape) != (n, 3):
        raise ValueError("means and scales must be [n, 3]")
    if tuple(scene.quats.shape) != (n, 4) or tuple(scene.opacities.shape) != (n,):
        raise ValueError("quats must be [n, 4] and opacities [n]")
    if tuple(scene.sh.shape) != (n, K, 3):
        raise ValueError(f"sh must be [n, {K}, 3] for sh_degree {sh_degree}, got {tuple(scene.sh.shape)}")


def _check_image_buffers(cam, fmt, image=None, state=None, last=None, n_contrib=None, dL=None):
    npx = int(cam.height) * int(cam.width)
    _need(image, npx * 3, "image")
    _need(state, npx, "state", STATE_BYTES[fmt])
    _need(last, npx, "last", 4)
    _need(n_contrib, npx, "n_contrib", 4)
    _need(dL, npx * 3, "dL_dimage")


def _check_grads(scene: "SceneTensors", grads: dict):
    for k, ref in zip(("means", "scales", "quats", "opacities", "sh"), scene.tensors()):
        if grads[k].shape != ref.shape:
            raise ValueError(f"grads[{k!r}] must have shape {tuple(ref.shape)}")


class Workspace:
    """Caller-owned device scratch for one stream (gs_workspace_size / _init)."""

    def __init__(self, n_cap: int, width_cap: int, height_cap: int, opts: RasterOpts | None = None,
                 device=None, stream=None, buffer: torch.Tensor | None = None):
        """`buffer` (uint8 CUDA tensor of at least required_bytes(...) + 256 bytes)
        lets a caller reuse one allocation for successive workspaces."""
        lib = _lib.load()
        opts = opts or RasterOpts()
        co = opts.to_c()
        self.nbytes = Workspace.required_bytes(n_cap, width_cap, height_cap, opts)
        dev = torch.device(device) if device is not None else torch.device("cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        if buffer is not None:
            if buffer.numel() < self.nbytes + 256 or buffer.device != self.device:
                raise ValueError("workspace buffer too small or on another device")
            self.buf = buffer
        else:
            self.buf = torch.empty(self.nbytes + 256, dtype=torch.uint8, device=self.device)
        base = (self.buf.data_ptr() + 255) & ~255
        self.c = _lib.GsWorkspace()
        with torch.cuda.device(self.device):
            st = stream if stream is not None else torch.cuda.current_stream(self.device)
            check(lib.gs_workspace_init(ctypes.byref(self.c), base, self.nbytes, n_cap, width_cap,
                                        height_cap, ctypes.byref(co), _stream(st)),
                  "gs_workspace_init")
        self.n_cap, self.width_cap, self.height_cap = n_cap, width_cap, height_cap
        self.pair_cap = int(self.c.pair_cap)

    @property
    def ref(self):
        return ctypes.byref(self.c)

    def sort_bytes(self) -> dict:
        """Sorting memory: depth-sort buffers and look-back words, pair buffers."""
        d, p = ctypes.c_size_t(0), ctypes.c_size_t(0)
        check(_lib.load().gs_workspace_sort_bytes(self.ref, ctypes.byref(d), ctypes.byref(p)),
              "gs_workspace_sort_bytes")
        return dict(depth_sort=int(d.value), pair_sort=int(p.value))

    def release_graph(self):
        """Frees the CUDA graph render_batch(graph=True) keeps for this workspace."""
        lib = _lib._lib
        if lib is not None:
            lib.gs_graph_release(ctypes.byref(self.c))

    def __del__(self):
        try:
            self.release_graph()
        except Exception:
            pass

    @staticmethod
    def required_bytes(n_cap: int, width_cap: int, height_cap: int, opts: RasterOpts | None = None) -> int:
        nbytes = ctypes.c_size_t(0)
        co = (opts or RasterOpts()).to_c()
        check(_lib.load().gs_workspace_size(n_cap, width_cap, height_cap, ctypes.byref(co),
                                            ctypes.byref(nbytes)), "gs_workspace_size")
        return int(nbytes.value)


def project(ws: Workspace, scene: SceneTensors, cam, opts: RasterOpts, stream=None):
    _check_scene(scene, opts.sh_degree)
    m, s, q, o, sh = scene.tensors()
    check(_lib.load().gs_project(ws.ref, _f32(m, "means"), _f32(s, "scales"), _f32(q, "quats"),
                                 _f32(o, "opacities"), _f32(sh, "sh"), scene.n,
                                 ctypes.byref(camera_to_c(cam)), ctypes.byref(opts.to_c()),
                                 _stream(stream)), "gs_project")


def sort(ws: Workspace, stream=None):
    check(_lib.load().gs_sort(ws.ref, _stream(stream)), "gs_sort")


def alloc_state(height: int, width: int, fmt: str, device) -> torch.Tensor:
    return torch.empty((height, width, STATE_BYTES[fmt]), dtype=torch.uint8, device=device)


def decode_state(state: torch.Tensor, fmt: str) -> torch.Tensor:
    """[H, W, 4] float32 (r, g, b, T) from a saved state of any format."""
    if fmt == "fp32":
        return state.view(torch.float32).clone()
    if fmt == "fp16":
        return state.view(torch.float16).float()
    if fmt == "unorm16":
        return (state.view(torch.int16).to(torch.int32) & 0xFFFF).float() / 65535.0
    return state.float() / 255.0


def raster_forward(ws: Workspace, cam, opts: RasterOpts, image=None, state=None, last=None,
                   n_contrib=None, want_image=True, want_n_contrib=False, stream=None):
    H, W = int(cam.height), int(cam.width)
    dev = ws.device
    if image is None and want_image:
        image = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    if state is None:
        state = alloc_state(H, W, opts.state_format, dev)
    if last is None:
        last = torch.empty((H, W), dtype=torch.int32, device=dev)
    if n_contrib is None and want_n_contrib:
        n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    _check_image_buffers(cam, opts.state_format, image, state, last, n_contrib)
    check(_lib.load().gs_raster_forward(ws.ref, ctypes.byref(camera_to_c(cam)),
                                        ctypes.byref(opts.to_c()), _f32(image, "image"),
                                        _ptr(state, "state"), _ptr(last, "last"),
                                        _ptr(n_contrib, "n_contrib"), _stream(stream)),
          "gs_raster_forward")
    return dict(image=image, state=state, last=last, n_contrib=n_contrib)


def bin(ws: Workspace, cam, opts: RasterOpts, stream=None):
    """First half of raster_forward: block lists of every visible splat's quad."""
    check(_lib.load().gs_bin(ws.ref, ctypes.byref(camera_to_c(cam)), ctypes.byref(opts.to_c()),
                             _stream(stream)), "gs_bin")


def blend_forward(ws: Workspace, cam, opts: RasterOpts, image, state, last, n_contrib=None,
                  stream=None):
    """Second half of raster_forward: front-to-back blending of the block lists."""
    _check_image_buffers(cam, opts.state_format, image, state, last, n_contrib)
    check(_lib.load().gs_blend_forward(ws.ref, ctypes.byref(camera_to_c(cam)),
                                       ctypes.byref(opts.to_c()), _f32(image, "image"),
                                       _ptr(state, "state"), _ptr(last, "last"),
                                       _ptr(n_contrib, "n_contrib"), _stream(stream)),
          "gs_blend_forward")


def blend_backward(ws: Workspace, cam, opts: RasterOpts, state, last, dL_dimage, stream=None):
    """First half of raster_backward: per-splat 2D gradients in the workspace."""
    _check_image_buffers(cam, opts.state_format, None, state, last, None, dL_dimage)
    check(_lib.load().gs_blend_backward(ws.ref, ctypes.byref(camera_to_c(cam)),
                                        ctypes.byref(opts.to_c()), _ptr(state, "state"),
                                        _ptr(last, "last"), _f32(dL_dimage, "dL_dimage"),
                                        _stream(stream)), "gs_blend_backward")


def project_backward(ws: Workspace, scene: SceneTensors, cam, opts: RasterOpts, grads: dict,
                     stream=None):
    """Second half of raster_backward: chain rule to the 3D parameters (added to grads)."""
    _check_scene(scene, opts.sh_degree)
    _check_grads(scene, grads)
    m, s, q, o, sh = scene.tensors()
    check(_lib.load().gs_project_backward(
        ws.ref, _f32(m, "means"), _f32(s, "scales"), _f32(q, "quats"), _f32(o, "opacities"),
        _f32(sh, "sh"), scene.n, ctypes.byref(camera_to_c(cam)), ctypes.byref(opts.to_c()),
        _f32(grads["means"], "d_means"), _f32(grads["scales"], "d_scales"),
        _f32(grads["quats"], "d_quats"), _f32(grads["opacities"], "d_opacities"),
        _f32(grads["sh"], "d_sh"), _stream(stream)), "gs_project_backward")
    return grads


def zero_grads(scene: SceneTensors) -> dict:
    return dict(means=torch.zeros_like(scene.means), scales=torch.zeros_like(scene.scales),
                quats=torch.zeros_like(scene.quats), opacities=torch.zeros_like(scene.opacities),
                sh=torch.zeros_like(scene.sh))


def raster_backward(ws: Workspace, scene: SceneTensors, cam, opts: RasterOpts, state, last,
                    dL_dimage, grads: dict | None = None, stream=None) -> dict:
    if grads is None:
        grads = zero_grads(scene)
    _check_scene(scene, opts.sh_degree)
    _check_grads(scene, grads)
    _check_image_buffers(cam, opts.state_format, None, state, last, None, dL_dimage)
    m, s, q, o, sh = scene.tensors()
    check(_lib.load().gs_raster_backward(
        ws.ref, _f32(m, "means"), _f32(s, "scales"), _f32(q, "quats"), _f32(o, "opacities"),
        _f32(sh, "sh"), scene.n, ctypes.byref(camera_to_c(cam)), ctypes.byref(opts.to_c()),
        _ptr(state, "state"), _ptr(last, "last"), _f32(dL_dimage, "dL_dimage"),
        _f32(grads["means"], "d_means"), _f32(grads["scales"], "d_scales"),
        _f32(grads["quats"], "d_quats"), _f32(grads["opacities"], "d_opacities"),
        _f32(grads["sh"], "d_sh"), _stream(stream)), "gs_raster_backward")
    return grads


def raster_forward_slab(ws: Workspace, cam, opts: RasterOpts, slab: int, n_slabs: int,
                        image=None, state=None, last=None, n_contrib=None, want_image=True,
                        want_n_contrib=False, stream=None):
    """Bins and blends depth slab `slab` of `n_slabs` alone (each pixel from
    T = 1): its colour C_k, state (C_k, T_k), last rank and count."""
    H, W = int(cam.height), int(cam.width)
    dev = ws.device
    if image is None and want_image:
        image = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    if state is None:
        state = alloc_state(H, W, opts.state_format, dev)
    if last is None:
        last = torch.empty((H, W), dtype=torch.int32, device=dev)
    if n_contrib is None and want_n_contrib:
        n_contrib = torch.empty((H, W), dtype=torch.int32, device=dev)
    _check_image_buffers(cam, opts.state_format, image, state, last, n_contrib)
    check(_lib.load().gs_raster_forward_slab(ws.ref, ctypes.byref(camera_to_c(cam)),
                                             ctypes.byref(opts.to_c()), int(slab), int(n_slabs),
                                             _f32(image, "image"), _ptr(state, "state"),
                                             _ptr(last, "last"), _ptr(n_contrib, "n_contrib"),
                                             _stream(stream)),
          "gs_raster_forward_slab")
    return dict(image=image, state=state, last=last, n_contrib=n_contrib)


def slab_composite(states: torch.Tensor, fmt: str, want_backward=True, stream=None) -> dict:
    """"Over" composite of slab states [n, H, W, bytes]: image [H, W, 3], trans
    [H, W] and, for the slabs' backward, t_front [n, H, W] and behind
    [n, H, W, 3]."""
    n, H, W = int(states.shape[0]), int(states.shape[1]), int(states.shape[2])
    if tuple(states.shape[3:]) != (STATE_BYTES[fmt],) or states.dtype != torch.uint8:
        raise ValueError(f"states must be uint8 [n, H, W, {STATE_BYTES[fmt]}]")
    dev = states.device
    image = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    trans = torch.empty((H, W), dtype=torch.float32, device=dev)
    t_front = torch.empty((n, H, W), dtype=torch.float32, device=dev) if want_backward else None
    behind = torch.empty((n, H, W, 3), dtype=torch.float32, device=dev) if want_backward else None
    check(_lib.load().gs_slab_composite(_ptr(states, "states"), STATE_FORMATS[fmt], n, H * W,
                                        _f32(image, "image"), _f32(trans, "trans"),
                                        _f32(t_front, "t_front"), _f32(behind, "behind"),
                                        _stream(stream)), "gs_slab_composite")
    return dict(image=image, trans=trans, t_front=t_front, behind=behind)


def raster_backward_slab(ws: Workspace, scene: SceneTensors, cam, opts: RasterOpts, slab: int,
                         n_slabs: int, state, last, dL_dimage, t_front=None, behind=None,
                         grads: dict | None = None, stream=None) -> dict:
    """Backward of one depth slab (after raster_forward_slab of that slab on ws):
    image gradient scaled by t_front [H, W], C' seeded with the slab's colour
    plus T_slab * behind [H, W, 3]; gradients added to `grads`."""
    if grads is None:
        grads = zero_grads(scene)
    _check_scene(scene, opts.sh_degree)
    _check_grads(scene, grads)
    _check_image_buffers(cam, opts.state_format, None, state, last, None, dL_dimage)
    H, W = int(cam.height), int(cam.width)
    _need(t_front, H * W, "t_front")
    _need(behind, H * W * 3, "behind")
    m, s, q, o, sh = scene.tensors()
    check(_lib.load().gs_raster_backward_slab(
        ws.ref, _f32(m, "means"), _f32(s, "scales"), _f32(q, "quats"), _f32(o, "opacities"),
        _f32(sh, "sh"), scene.n, ctypes.byref(camera_to_c(cam)), ctypes.byref(opts.to_c()),
        int(slab), int(n_slabs), _ptr(state, "state"), _ptr(last, "last"),
        _f32(t_front, "t_front"), _f32(behind, "behind"), _f32(dL_dimage, "dL_dimage"),
        _f32(grads["means"], "d_means"), _f32(grads["scales"], "d_scales"),
        _f32(grads["quats"], "d_quats"), _f32(grads["opacities"], "d_opacities"),
        _f32(grads["sh"], "d_sh"), _stream(stream)), "gs_raster_backward_slab")
    return grads


def zero_touched_gradients(ws: Workspace, grads: dict, stream=None) -> dict:
    """Zeroes the gradient rows of the splats the last sort on ws ordered (the
    rows a backward on that view adds to); buffers that were all zero before
    that backward are all zero again.  Call before the next sort on ws."""
    n = int(grads["means"].shape[0])
    K = (int(ws.c.sh_degree) + 1) ** 2
    shapes = dict(means=(n, 3), scales=(n, 3), quats=(n, 4), opacities=(n,), sh=(n, K, 3))
    for k, shp in shapes.items():
        if tuple(grads[k].shape) != shp:
            raise ValueError(f"grads[{k!r}] must have shape {shp}")
    check(_lib.load().gs_zero_touched_gradients(
        ws.ref, n, _f32(grads["means"], "d_means"), _f32(grads["scales"], "d_scales"),
        _f32(grads["quats"], "d_quats"), _f32(grads["opacities"], "d_opacities"),
        _f32(grads["sh"], "d_sh"), _stream(stream)), "gs_zero_touched_gradients")
    return grads


def loss(image, target, kind: str = "l2", dL_dimage=None, loss_out=None, stream=None):
    """Summed L1 / L2 loss; returns (dL_dimage, loss as a 1-element float64 tensor)."""
    if dL_dimage is None:
        dL_dimage = torch.empty_like(image)
    if loss_out is None:
        loss_out = torch.empty(1, dtype=torch.float64, device=image.device)
    if target.numel() != image.numel() or dL_dimage.numel() != image.numel():
        raise ValueError("image, target and dL_dimage must have the same size")
    if loss_out.dtype != torch.float64:
        raise ValueError("loss_out must be float64")
    k = {"l1": GS_LOSS_L1, "l2": GS_LOSS_L2}[kind]
    check(_lib.load().gs_loss(_f32(image, "image"), _f32(target, "target"), image.numel(), k,
                              _f32(dL_dimage, "dL_dimage"), _ptr(loss_out, "loss"),
                              _stream(stream)), "gs_loss")
    return dL_dimage, loss_out


def render(ws: Workspace, scene: SceneTensors, cam, opts: RasterOpts, stream=None, **kw):
    """project -> sort -> raster_forward."""
    project(ws, scene, cam, opts, stream)
    sort(ws, stream)
    return raster_forward(ws, cam, opts, stream=stream, **kw)


def fp32_fma_rate(iters: int = 1 << 16, stream=None) -> float:
    """Measured FP32 FMA rate of the current GPU in TFLOP/s (a measurement helper)."""
    out = ctypes.c_double(0.0)
    check(_lib.load().gs_fp32_fma_rate(int(iters), ctypes.byref(out), _stream(stream)),
          "gs_fp32_fma_rate")
    return float(out.value)


def check_status(ws: Workspace, stream=None):
    check(_lib.load().gs_check_status(ws.ref, _stream(stream)), "gs_check_status")


def read_counters(ws: Workspace, stream=None) -> dict:
    out = (ctypes.c_int64 * 6)()
    check(_lib.load().gs_read_counters(ws.ref, out, _stream(stream)), "gs_read_counters")
    return dict(visible=int(out[0]), pairs=int(out[1]), status=int(out[2]), blocks=int(out[3]),
                pairs_wanted=int(out[4]), live_pairs=int(out[5]))


_ARRAY_DTYPES = {
    _lib.GS_ARRAY_SORTED_IDS: (torch.int32, 1), _lib.GS_ARRAY_DEPTH_KEYS: (torch.int32, 1),
    _lib.GS_ARRAY_RECORDS: (torch.float32, 12), _lib.GS_ARRAY_PAIR_BLOCKS: (torch.int32, 1),
    _lib.GS_ARRAY_PAIR_RANKS: (torch.int32, 1), _lib.GS_ARRAY_RANGES: (torch.int32, 2),
    _lib.GS_ARRAY_GRAD2D: (torch.float32, 12), _lib.GS_ARRAY_BOXES: (torch.int32, 2),
}


def copy_array(ws: Workspace, which: int, count: int, stream=None) -> torch.Tensor:
    dt, w = _ARRAY_DTYPES[which]
    out = torch.empty((count, w) if w > 1 else (count,), dtype=dt, device=ws.device)
    check(_lib.load().gs_copy_array(ws.ref, which, _ptr(out), out.numel() * 4, _stream(stream)),
          "gs_copy_array")
    return out


def sort_pairs(ws: Workspace, keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32,
               stream=None):
    """Stable radix sort of (u32 key, u32 value) pairs given as int32 tensors."""
    if keys.dtype != torch.int32 or vals.dtype != torch.int32 or keys.numel() != vals.numel():
        raise ValueError("keys and vals must be int32 tensors of the same size")
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    check(_lib.load().gs_sort_pairs(ws.ref, _ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo),
                                    keys.numel(), key_bits, _stream(stream)), "gs_sort_pairs")
    return ko, vo


def sort_pairs_noalloc(keys: torch.Tensor, vals: torch.Tensor, key_bits: int = 32, stream=None):
    """Same sort as sort_pairs, for callers that cannot hand the library any
    scratch memory: the library keeps a fixed array of its own (at most
    GS_SORT_NOALLOC_MAX_PAIRS pairs; calls overlapping on the GPU race)."""
    if keys.dtype != torch.int32 or vals.dtype != torch.int32 or keys.numel() != vals.numel():
        raise ValueError("keys and vals must be int32 tensors of the same size")
    if keys.device != vals.device:
        raise ValueError("keys and vals must be on the same device")
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    with torch.cuda.device(keys.device):   # the library uses the current device's array
        check(_lib.load().gs_sort_pairs_noalloc(_ptr(keys), _ptr(vals), _ptr(ko), _ptr(vo),
                                                keys.numel(), key_bits, _stream(stream)),
              "gs_sort_pairs_noalloc")
    return ko, vo


def sort_pairs_noalloc_status(device=None, stream=None):
    """Raises GsError(GS_ERR_TIMEOUT) when a look-back wait of the last
    sort_pairs_noalloc on `device` gave up (synchronises the stream)."""
    with torch.cuda.device(device if device is not None else torch.cuda.current_device()):
        check(_lib.load().gs_sort_pairs_noalloc_status(_stream(stream)),
              "gs_sort_pairs_noalloc_status")


def stalled_sort_selftest(ws, keys: torch.Tensor, vals: torch.Tensor, spin_limit: int, stream=None):
    """Self-test of the bounded device waits: one radix pass with tile 0
    withheld, so its look-back waits give up after `spin_limit` polls and the
    device status reads GS_ERR_TIMEOUT.  ws None: the allocation-free sort's
    array.  Returns the (wrong) output tensors."""
    if keys.dtype != torch.int32 or vals.dtype != torch.int32 or keys.numel() != vals.numel():
        raise ValueError("keys and vals must be int32 tensors of the same size")
    ko, vo = torch.empty_like(keys), torch.empty_like(vals)
    with torch.cuda.device(keys.device):
        check(_lib.load().gs_test_stalled_sort(ws.ref if ws is not None else None, _ptr(keys),
                                               _ptr(vals), _ptr(ko), _ptr(vo), keys.numel(),
                                               int(spin_limit), _stream(stream)),
              "gs_test_stalled_sort")
    return ko, vo


@dataclass
class Request:
    """One gs_render_batch request (tensors must outlive the call's GPU work)."""
    scene: SceneTensors
    camera: object
    opts: RasterOpts
    backward: bool = False
    loss_kind: str | None = None
    target: torch.Tensor | None = None
    dL_dimage: torch.Tensor | None = None
    outputs: dict = field(default_factory=dict)
    zero_touched: int = 0   # 1: zero the previous view's gradient rows first; 2: grads = this view's alone
    loss_host: torch.Tensor | None = None       # pinned float64 [1]: the loss copied there too


def render_batch(requests, ws: Workspace, stream=None, graph: bool = False):
    """Allocates each request's outputs, then runs all requests in one C call
    (`graph`: as one CUDA graph, gs_render_batch_graph; needs a non-default stream)."""
    lib = _lib.load()
    arr = (_lib.GsRequest * len(requests))()
    for i, rq in enumerate(requests):
        H, W = int(rq.camera.height), int(rq.camera.width)
        dev = ws.device
        out = rq.outputs
        # outputs the caller did not provide are allocated (only then)
        if "image" not in out:
            out["image"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
        if "state" not in out:
            out["state"] = alloc_state(H, W, rq.opts.state_format, dev)
        if "last" not in out:
            out["last"] = torch.empty((H, W), dtype=torch.int32, device=dev)
        sc = rq.scene
        _check_scene(sc, rq.opts.sh_degree)
        _check_image_buffers(rq.camera, rq.opts.state_format, out["image"], out["state"], out["last"],
                             out.get("n_contrib"), rq.dL_dimage if rq.backward and not rq.loss_kind else None)
        if rq.backward and rq.loss_kind:
            _need(rq.target, H * W * 3, "target")
        c = arr[i]
        c.scene.means, c.scene.scales, c.scene.quats = _ptr(sc.means), _ptr(sc.scales), _ptr(sc.quats)
        c.scene.opacities, c.scene.sh = _ptr(sc.opacities), _ptr(sc.sh)
        c.scene.n, c.scene.sh_degree = sc.n, sc.sh_degree
        c.camera = camera_to_c(rq.camera)
        c.opts = rq.opts.to_c()
        c.mode = GS_MODE_FORWARD_BACKWARD if rq.backward else GS_MODE_FORWARD
        c.image, c.state, c.last = _ptr(out["image"]), _ptr(out["state"]), _ptr(out["last"])
        c.n_contrib = _ptr(out.get("n_contrib"))
        if rq.backward:
            if rq.loss_kind:
                c.loss_kind = {"l1": GS_LOSS_L1, "l2": GS_LOSS_L2}[rq.loss_kind]
                c.target = _ptr(rq.target)
                if "dL_dimage" not in out:
                    out["dL_dimage"] = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
                if "loss" not in out:
                    out["loss"] = torch.empty(1, dtype=torch.float64, device=dev)
                c.dL_dimage, c.loss = _ptr(out["dL_dimage"]), _ptr(out["loss"])
            else:
                c.loss_kind = GS_LOSS_NONE
                c.dL_dimage = _ptr(rq.dL_dimage)
            if "grads" not in out:
                out["grads"] = zero_grads(sc)
            g = out["grads"]
            _check_grads(sc, g)
            c.d_means, c.d_scales, c.d_quats = _ptr(g["means"]), _ptr(g["scales"]), _ptr(g["quats"])
            c.d_opacities, c.d_sh = _ptr(g["opacities"]), _ptr(g["sh"])
            c.zero_touched = int(rq.zero_touched)
            if rq.loss_host is not None:
                if rq.loss_host.is_cuda or not rq.loss_host.is_pinned() or \
                        rq.loss_host.dtype != torch.float64 or rq.loss_host.numel() < 1:
                    raise ValueError("loss_host must be a pinned float64 host tensor")
                c.loss_host = rq.loss_host.data_ptr()
    if graph:
        check(lib.gs_render_batch_graph(arr, len(requests), ws.ref, _stream(stream)),
              "gs_render_batch_graph")
    else:
        check(lib.gs_render_batch(arr, len(requests), ws.ref, _stream(stream)), "gs_render_batch")
    return requests


__all__ = ["RasterOpts", "SceneTensors", "Workspace", "project", "sort", "raster_forward", "bin",
           "blend_forward", "blend_backward", "project_backward",
           "raster_backward", "loss", "render", "render_batch", "Request", "check_status",
           "read_counters", "fp32_fma_rate", "copy_array", "sort_pairs", "sort_pairs_noalloc", "sort_pairs_noalloc_status", "stalled_sort_selftest", "decode_state", "alloc_state",
           "camera_to_c", "GsError", "zero_grads", "NONE_RANK", "raster_forward_slab",
           "slab_composite", "raster_backward_slab"]
