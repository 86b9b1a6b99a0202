"""torch.autograd wrapper of the rasterizer.

GSRender.apply(means, scales, quats, opacities, sh, camera, opts, workspace)
renders one view with gs_project / gs_sort / gs_raster_forward and, in the
backward pass, calls gs_raster_backward: the forward's per-pixel state (stored
colour and transmittance, last-fragment rank) is saved, alpha is recomputed,
and no per-fragment data is kept (Procedure 1).

A workspace holds the sorted splats and block lists of the last view it
rendered.  The Function remembers the workspace generation it rendered with;
if another view reused the workspace before this one's backward runs, the
backward first redoes projection, sort and binning for its own view.

`render_activated` applies the usual parameter activations in PyTorch
(scales = exp(log_scales), opacity = sigmoid(logit)); the rasterizer itself
takes activated values.
"""
from __future__ import annotations

import torch

from . import (RasterOpts, SceneTensors, Workspace, bin, blend_backward, blend_forward,
               project, project_backward, sort, alloc_state, zero_grads)


class _Generation:
    """Per-workspace counter of rendered views (host side)."""

    @staticmethod
    def bump(ws: Workspace) -> int:
        ws._generation = getattr(ws, "_generation", 0) + 1
        return ws._generation

    @staticmethod
    def current(ws: Workspace) -> int:
        return getattr(ws, "_generation", 0)


def _prepare(ws, scene, cam, opts):
    project(ws, scene, cam, opts)
    sort(ws)
    bin(ws, cam, opts)


class GSRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, camera, opts: RasterOpts,
                ws: Workspace):
        scene = SceneTensors(means.detach().contiguous(), scales.detach().contiguous(),
                             quats.detach().contiguous(), opacities.detach().contiguous(),
                             sh.detach().contiguous(), opts.sh_degree)
        H, W = int(camera.height), int(camera.width)
        image = torch.empty((H, W, 3), dtype=torch.float32, device=means.device)
        state = alloc_state(H, W, opts.state_format, means.device)
        last = torch.empty((H, W), dtype=torch.int32, device=means.device)
        _prepare(ws, scene, camera, opts)
        blend_forward(ws, camera, opts, image, state, last)
        ctx.generation = _Generation.bump(ws)
        ctx.scene, ctx.camera, ctx.opts, ctx.ws = scene, camera, opts, ws
        ctx.save_for_backward(state, last)
        ctx.mark_non_differentiable(state, last)
        return image, state, last

    @staticmethod
    def backward(ctx, d_image, d_state=None, d_last=None):
        state, last = ctx.saved_tensors
        ws, scene, cam, opts = ctx.ws, ctx.scene, ctx.camera, ctx.opts
        if _Generation.current(ws) != ctx.generation:
            _prepare(ws, scene, cam, opts)   # the workspace served another view since
            _Generation.bump(ws)
            ctx.generation = _Generation.current(ws)
        if d_image is None:
            d_image = torch.zeros((cam.height, cam.width, 3), dtype=torch.float32,
                                  device=state.device)
        grads = zero_grads(scene)
        blend_backward(ws, cam, opts, state, last, d_image.contiguous().float())
        project_backward(ws, scene, cam, opts, grads)
        return (grads["means"], grads["scales"], grads["quats"], grads["opacities"], grads["sh"],
                None, None, None)


def render(means, scales, quats, opacities, sh, camera, opts: RasterOpts, ws: Workspace):
    """Differentiable render of one view; returns the [H, W, 3] image."""
    image, _, _ = GSRender.apply(means, scales, quats, opacities, sh, camera, opts, ws)
    return image


def render_activated(means, log_scales, quats, opacity_logits, sh, camera, opts: RasterOpts,
                     ws: Workspace):
    """render() on raw parameters: scales = exp(log_scales), opacity = sigmoid(logits)."""
    return render(means, torch.exp(log_scales), quats, torch.sigmoid(opacity_logits), sh, camera,
                  opts, ws)


class Renderer(torch.nn.Module):
    """Splat scene as trainable parameters (raw, pre-activation) plus a workspace."""

    def __init__(self, scene_np, width_cap: int, height_cap: int, opts: RasterOpts | None = None,
                 device="cuda"):
        super().__init__()
        import numpy as np

        def p(a):
            return torch.nn.Parameter(torch.as_tensor(np.asarray(a), dtype=torch.float32,
                                                      device=device).contiguous())
        self.means = p(scene_np.means)
        self.log_scales = p(np.log(scene_np.scales))
        self.quats = p(scene_np.quats)
        o = np.clip(scene_np.opacities.astype(np.float64), 1e-6, 1 - 1e-6)
        self.opacity_logits = p(np.log(o / (1 - o)))
        self.sh = p(scene_np.sh)
        self.opts = opts or RasterOpts(sh_degree=scene_np.sh_degree)
        self.ws = Workspace(scene_np.n, width_cap, height_cap, self.opts, device=device)

    def forward(self, camera):
        return render_activated(self.means, self.log_scales, self.quats, self.opacity_logits,
                                self.sh, camera, self.opts, self.ws)
