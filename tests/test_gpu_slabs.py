"""Depth slabs through the C ABI: each slab of the depth order is rendered on
its own (from T = 1), the "over" composite of the slabs' (C_k, T_k) is the
single-pass image, and the slabs' backward calls (image gradient scaled by the
transmittance in front, C' seeded with the colour behind) sum to the
single-pass gradient.  One workspace per slab, as one GPU per slab would hold
(here all on one GPU, run one after another)."""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_18764_gb300 as gs
import synthetic as syn
from gpu_helpers import AMBIG_IMAGE, GROUPS, oracle_opts, rel_l2

pytestmark = pytest.mark.gpu


def _slab_render(scene_np, cam, opts, n_slabs):
    scene = gs.SceneTensors.from_numpy(scene_np)
    H, W = cam.height, cam.width
    states = torch.empty((n_slabs, H, W, gs.STATE_BYTES[opts.state_format]), dtype=torch.uint8,
                         device="cuda")
    slabs = []
    for k in range(n_slabs):
        ws = gs.Workspace(scene.n, W, H, opts)
        gs.project(ws, scene, cam, opts)
        gs.sort(ws)
        out = gs.raster_forward_slab(ws, cam, opts, k, n_slabs, state=states[k], want_n_contrib=True)
        gs.check_status(ws)
        slabs.append((ws, out))
    comp = gs.slab_composite(states, opts.state_format)
    torch.cuda.synchronize()
    return scene, states, slabs, comp


@pytest.mark.parametrize("n_slabs", [1, 2, 3, 5])
def test_slabs_composite_to_the_single_pass_image(n_slabs):
    scene_np = syn.cube_scene(3000, seed=81, sh_degree=2, log_scale_mean=-2.6)
    cam = syn.look_at((0.4, -0.3, -3.4), (0.0, 0.0, 0.0), 50.0, 101, 83)
    opts = gs.RasterOpts(sh_degree=2, t_cull=0.0)
    scene, states, slabs, comp = _slab_render(scene_np, cam, opts, n_slabs)
    ref = oracle.render(scene_np, cam, oracle_opts(opts, cam))
    ok = (ref["ambig"] & AMBIG_IMAGE) == 0
    img = comp["image"].cpu().numpy().astype(np.float64)
    err = np.abs(img - ref["color"]).max(axis=2)
    assert err[ok].max() <= 1e-4, f"composite max-abs {err[ok].max():.2e}"
    assert np.abs(comp["trans"].cpu().numpy() - ref["T"])[ok].max() <= 1e-5
    # every fragment is in exactly one slab
    total = sum(out["n_contrib"].cpu().numpy().astype(np.int64) for _, out in slabs)
    np.testing.assert_array_equal(total[ok], ref["nfrag"][ok])
    # and the single-pass render agrees to FP32 reassociation
    single = gs.render(gs.Workspace(scene.n, cam.width, cam.height, opts), scene, cam, opts)
    assert torch.max(torch.abs(single["image"] - comp["image"])).item() <= 2e-6
    print(f"{n_slabs} slabs: composite max-abs {err[ok].max():.2e} vs the oracle")


@pytest.mark.parametrize("n_slabs,order", [(2, "front_to_back"), (3, "front_to_back"),
                                           (3, "back_to_front")])
def test_slab_gradients_sum_to_the_single_pass(n_slabs, order):
    scene_np = syn.cube_scene(2500, seed=82, sh_degree=1, log_scale_mean=-2.4)
    cam = syn.look_at((0.0, 0.2, -3.3), (0.0, 0.0, 0.0), 50.0, 96, 80)
    opts = gs.RasterOpts(sh_degree=1, t_cull=0.0, backward_order=order)
    oo = oracle_opts(opts, cam)
    clean = (oracle.render(scene_np, cam, oo)["ambig"] & AMBIG_IMAGE) == 0
    g = syn.uniform_image(cam.height, cam.width, seed=83, lo=-1.0, hi=1.0) * clean[..., None]
    gt = torch.from_numpy(g.astype(np.float32)).cuda()
    scene, states, slabs, comp = _slab_render(scene_np, cam, opts, n_slabs)
    grads = gs.zero_grads(scene)
    for k, (ws, out) in enumerate(slabs):
        gs.raster_backward_slab(ws, scene, cam, opts, k, n_slabs, states[k], out["last"], gt,
                                t_front=comp["t_front"][k], behind=comp["behind"][k], grads=grads)
        gs.check_status(ws)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    ref = oracle.backward(scene_np, cam, g.astype(np.float64), oo)
    errs = {k: rel_l2(got[k], ref[k]) for k in GROUPS}
    print(f"{n_slabs} slabs ({order}): gradient rel-L2 vs the oracle {errs}")
    for k, e in errs.items():
        assert e <= 1e-3, f"{k}: {e:.3e}"
    # against the single-pass CUDA backward
    ws1 = gs.Workspace(scene.n, cam.width, cam.height, opts)
    out1 = gs.render(ws1, scene, cam, opts)
    g1 = gs.raster_backward(ws1, scene, cam, opts, out1["state"], out1["last"], gt)
    for k in GROUPS:
        assert rel_l2(got[k], g1[k].cpu().numpy().astype(np.float64)) <= 1e-5, k


def test_slab_arguments_are_checked():
    scene_np, cam, _ = syn.tiny_scene_1k()
    opts = gs.RasterOpts()
    scene = gs.SceneTensors.from_numpy(scene_np)
    ws = gs.Workspace(scene.n, cam.width, cam.height, opts)
    gs.project(ws, scene, cam, opts)
    gs.sort(ws)
    for k, n in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(gs.GsError) as e:
            gs.raster_forward_slab(ws, cam, opts, k, n)
        assert e.value.code == gs._lib.GS_ERR_INVALID_ARG
    chunked = gs.RasterOpts(chunked=1, pair_capacity=1 << 16)
    wsc = gs.Workspace(scene.n, cam.width, cam.height, chunked)
    gs.project(wsc, scene, cam, chunked)
    with pytest.raises(gs.GsError):
        gs.raster_forward_slab(wsc, cam, chunked, 0, 2)
