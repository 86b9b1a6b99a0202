"""Full-size parity: the 3.0M-splat 1256x828 view in the launch configuration
the benchmark times (FP32 state, t_cull 1e-4, block reduction), checked on
sampled outputs the oracle computes one by one: pixels (colour, transmittance,
fragment count, last fragment) and the complete gradients of sampled splats."""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_18764_gb300 as gs
import synthetic as syn
from gpu_helpers import AMBIG_IMAGE, GROUPS, last_ids, oracle_opts, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_view():
    assert torch.cuda.is_available()
    from paper_2505_18764_gb300 import build
    build.build_library()
    scene_np, cam, _ = syn.mipnerf_scene_3m()
    opts = gs.RasterOpts(state_format="fp32", sh_degree=3, t_cull=1e-4)
    scene = gs.SceneTensors.from_numpy(scene_np)
    ws = gs.Workspace(scene.n, cam.width, cam.height, opts)
    out = gs.render(ws, scene, cam, opts, want_n_contrib=True)
    g = syn.uniform_image(cam.height, cam.width, seed=202, lo=-1.0, hi=1.0)
    grads = gs.raster_backward(ws, scene, cam, opts, out["state"], out["last"],
                               torch.from_numpy(g).cuda())
    gs.check_status(ws)
    torch.cuda.synchronize()
    return dict(scene_np=scene_np, cam=cam, opts=opts, ws=ws, out=out, g=g,
                grads={k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()})


def test_fullsize_sampled_pixels(full_view):
    v = full_view
    cam = v["cam"]
    rng = np.random.default_rng(301)
    pix = rng.choice(cam.width * cam.height, size=384, replace=False).astype(np.int32)
    ref = oracle.render(v["scene_np"], cam, oracle_opts(v["opts"], cam), pixels=pix)
    ok = (ref["ambig"] & AMBIG_IMAGE) == 0
    assert ok.sum() >= 200, f"only {ok.sum()} clean pixels"
    img = v["out"]["image"].cpu().numpy().reshape(-1, 3)[pix].astype(np.float64)
    err = np.abs(img - ref["color"]).max(axis=1)
    assert err[ok].max() <= 1e-4, f"image max-abs {err[ok].max():.3e}"
    nc = v["out"]["n_contrib"].cpu().numpy().reshape(-1)[pix]
    np.testing.assert_array_equal(nc[ok], ref["nfrag"][ok])
    T = gs.decode_state(v["out"]["state"], "fp32")[..., 3].cpu().numpy().reshape(-1)[pix]
    assert np.abs(T - ref["T"])[ok].max() <= 1e-5
    np.testing.assert_array_equal(last_ids(v["ws"], v["out"]).reshape(-1)[pix][ok], ref["last"][ok])
    print(f"clean pixels {ok.sum()}/384, mean fragments {ref['nfrag'].mean():.1f}, "
          f"max-abs {err[ok].max():.2e}")


def _stratified_splats(ws, rng, per_stratum=16):
    """Depth ranks of sampled splats in three strata: large footprints (boxes
    over 8 blocks, at most 36), splats on the 20 longest block lists (the
    blocks walked by 8x4 and 4x4 footprints at the default split threshold;
    taken from the first 256 entries of each list, which are not T-culled
    everywhere), and the rest (boxes of at most 8 blocks)."""
    V = gs.read_counters(ws)["visible"]
    boxes = gs.copy_array(ws, gs._lib.GS_ARRAY_BOXES, V).cpu().numpy().astype(np.int64)
    nblk = (boxes[:, 1] & 0xFFFF) * (boxes[:, 1] >> 16)
    big = rng.choice(np.where((nblk > 8) & (nblk <= 36))[0], size=per_stratum, replace=False)
    nb = gs.read_counters(ws)["blocks"]
    ranges = gs.copy_array(ws, gs._lib.GS_ARRAY_RANGES, nb).cpu().numpy().astype(np.int64)
    ranges = ranges.reshape(-1, 2) & 0xFFFFFFFF
    lens = ranges[:, 1] - ranges[:, 0]
    longest = np.argsort(-lens, kind="stable")[:20]
    live = gs.read_counters(ws)["live_pairs"]
    pair_ranks = gs.copy_array(ws, gs._lib.GS_ARRAY_PAIR_RANKS, live).cpu().numpy().astype(np.int64)
    on_long = np.unique(np.concatenate([pair_ranks[b:min(b + 256, e)] for b, e in ranges[longest]]))
    on_long = np.setdiff1d(on_long, big)
    dense = rng.choice(on_long, size=per_stratum, replace=False)
    rest = np.setdiff1d(np.where(nblk <= 8)[0], np.concatenate([big, dense]))
    other = rng.choice(rest, size=per_stratum, replace=False)
    return dict(large=big, long_lists=dense, other=other), int(lens[longest[-1]])


def test_fullsize_sampled_splat_gradients(full_view):
    """Complete gradients of 48 sampled splats at the benchmark's size and launch
    configuration, stratified by footprint, against the oracle one splat at a
    time (each traced over its own pixels)."""
    v = full_view
    cam = v["cam"]
    ws = v["ws"]
    V = gs.read_counters(ws)["visible"]
    ids = gs.copy_array(ws, gs._lib.GS_ARRAY_SORTED_IDS, V).cpu().numpy()
    strata, shortest_long = _stratified_splats(ws, np.random.default_rng(302))
    assert shortest_long >= gs._lib.GS_SPLIT_THRESHOLD_DEFAULT   # those blocks take split footprints
    pick = ids[np.concatenate(list(strata.values()))]
    ref = oracle.splat_grads(v["scene_np"], cam, v["g"].astype(np.float64), pick,
                             oracle_opts(v["opts"], cam))
    lo = 0
    for name, ranks in strata.items():
        sl = slice(lo, lo + len(ranks))
        lo += len(ranks)
        errs = {k: rel_l2(v["grads"][k][pick[sl]], ref[k][sl]) for k in GROUPS}
        print(f"{name}: {len(ranks)} splats, {int(ref['pixels'][sl].sum())} traced pixels, "
              f"gradient rel-L2 {errs}")
        assert np.linalg.norm(ref["opacities"][sl]) > 0.0, name
        for k, e in errs.items():
            assert e <= 1e-3, f"{name} {k}: {e:.3e}"
