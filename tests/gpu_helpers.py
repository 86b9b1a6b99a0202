"""Shared helpers for the GPU parity tests (CUDA path via the C ABI vs the oracle)."""
import numpy as np
import torch

import oracle
import paper_2505_18764_gb300 as gs

# Oracle tie-band bits that make a pixel's image or coverage ambiguous between
# FP32 and FP64 evaluation: 1 alpha cutoff, 2 depth tie, 4 T-cull, 8 near plane.
AMBIG_IMAGE = 1 | 2 | 4 | 8

GROUPS = ("means", "scales", "quats", "opacities", "sh")


def cut_band(cam) -> float:
    """Tie band on |power - ln(1/(255 o))| for this image size.  The FP32 centre
    mu_2D carries ~2e-7 * (image size) px of rounding error, which moves power by
    up to ~3/sigma times that (sigma >= 0.55 px after the 0.3 dilation); the band
    is about 5x that bound, and never below 5e-4."""
    return max(5e-4, 3e-6 * max(int(cam.width), int(cam.height)))


def oracle_opts(opts: gs.RasterOpts, cam=None, **kw):
    clamp = opts.state_format in ("unorm16", "unorm8")
    if cam is not None and "band_cut" not in kw:
        kw["band_cut"] = cut_band(cam)
    return oracle.opts_array(t_cull=opts.t_cull, clamp01=clamp, **kw)


def run_forward(scene_np, cam, opts, n_contrib=True):
    scene = gs.SceneTensors.from_numpy(scene_np)
    ws = gs.Workspace(max(scene.n, 1), cam.width, cam.height, opts)
    out = gs.render(ws, scene, cam, opts, want_n_contrib=n_contrib)
    gs.check_status(ws)
    return scene, ws, out


def run_forward_backward(scene_np, cam, opts, g):
    scene, ws, out = run_forward(scene_np, cam, opts)
    gt = torch.as_tensor(g, dtype=torch.float32).contiguous().cuda()
    grads = gs.raster_backward(ws, scene, cam, opts, out["state"], out["last"], gt)
    gs.check_status(ws)
    torch.cuda.synchronize()
    return scene, ws, out, {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def last_ids(ws, out):
    """Map the GPU's per-pixel last depth rank to a splat index (-1 for none)."""
    V = gs.read_counters(ws)["visible"]
    ids = gs.copy_array(ws, gs._lib.GS_ARRAY_SORTED_IDS, max(V, 1)).cpu().numpy()
    last = out["last"].cpu().numpy().astype(np.int64) & 0xFFFFFFFF
    res = np.full(last.shape, -1, dtype=np.int64)
    has = last != gs.NONE_RANK
    res[has] = ids[last[has]]
    return res
