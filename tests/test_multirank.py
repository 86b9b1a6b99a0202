"""Multi-rank host logic on CPU ranks (gloo, world size 2).

* Replicas: the benchmark's per-rank view assignment and its max-over-ranks
  elapsed time, run through torch.distributed exactly as under torchrun.
* Depth slabs: the compositing algebra a depth-sharded renderer would rely on.
  With the globally depth-sorted splats split into a front and a back slab,
  each rank renders its own slab; one all-gather of per-pixel (C, T) and the
  "over" operator C = C_f + T_f C_b, T = T_f T_b give the full image.  The
  backward needs one exchange back: the back slab's splats see the image
  gradient T_f g, the front slab's see g plus the effect of T_f on the back
  slab's colour, d(sum_p (g . C_b) T_f) / dtheta_f.  Since sum_i T_i alpha_i =
  1 - T_final (Eq. 2), T_f = 1 - (the front slab rendered in colour 1), so
  that term is minus the gradient of a white render weighted by g . C_b.
  Both are checked against the FP64 oracle's full render and backward
  (t_cull = 0: a slab does not know the transmittance in front of it).
"""
from __future__ import annotations

import math
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthetic as syn  # noqa: E402

WORLD = 2
_Y00 = 0.5 / math.sqrt(math.pi)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)


def _spawn(fn, *args):
    port = _free_port()
    mp.start_processes(fn, args=(WORLD, port) + args, nprocs=WORLD, join=True,
                       start_method="spawn")


# ---------------------------------------------------------------------------
# replicas
# ---------------------------------------------------------------------------
def _replica_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import bench
    _init(rank, world, port)
    try:
        angles = [None] * world
        dist.all_gather_object(angles, bench.replica_orbit_angle(rank, world))
        # ranks report different elapsed times; the job's time is the slowest
        mine = 10.0 + 7.5 * rank
        job = bench.max_over_ranks_ms(mine, torch.device("cpu"), world)
        np.save(os.path.join(out_dir, f"replica_{rank}.npy"), np.array(angles + [job]))
    finally:
        dist.destroy_process_group()


def test_replica_views_and_max_over_ranks(tmp_path):
    _spawn(_replica_worker, str(tmp_path))
    r0 = np.load(tmp_path / "replica_0.npy")
    r1 = np.load(tmp_path / "replica_1.npy")
    np.testing.assert_array_equal(r0, r1)
    angles, job = r0[:WORLD], r0[WORLD]
    assert len(set(angles.tolist())) == WORLD          # every rank its own view
    np.testing.assert_allclose(angles, 2 * math.pi * np.arange(WORLD) / WORLD)
    assert job == 17.5                                  # the slowest rank's time


# ---------------------------------------------------------------------------
# depth slabs
# ---------------------------------------------------------------------------
def _slab_scene():
    scene = syn.cube_scene(192, seed=31, sh_degree=1, log_scale_mean=-2.2)
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 50.0, 48, 40)
    g = np.random.default_rng(7).uniform(-1.0, 1.0, (cam.height, cam.width, 3))
    return scene, cam, g


def _slab_ids(scene, cam, rank, world):
    order = oracle.depth_order(scene, cam)          # visible splats, front to back
    cuts = np.linspace(0, order.shape[0], world + 1).astype(int)
    return np.sort(order[cuts[rank]:cuts[rank + 1]])


def _white(scene):
    w = scene.subset(np.arange(scene.n))
    w.sh[:] = 0.0
    w.sh[:, 0, :] = np.float32(0.5 / _Y00)        # colour 1 in every channel
    return w


def _slab_worker(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    _init(rank, world, port)
    try:
        scene, cam, g = _slab_scene()
        opts = oracle.opts_array(t_cull=0.0)
        ids = _slab_ids(scene, cam, rank, world)
        mine = scene.subset(ids)
        r = oracle.render(mine, cam, opts)
        ct = torch.from_numpy(np.concatenate([r["color"], r["T"][..., None]], axis=-1))
        gathered = [torch.zeros_like(ct) for _ in range(world)]
        dist.all_gather(gathered, ct)
        C = np.zeros_like(r["color"])
        T = np.ones_like(r["T"])
        for k in range(world):                      # front to back "over"
            C = C + T[..., None] * gathered[k][..., :3].numpy()
            T = T * gathered[k][..., 3].numpy()
        # backward: transmittance in front of this slab and colour behind it
        T_front = np.ones_like(T)
        for k in range(rank):
            T_front = T_front * gathered[k][..., 3].numpy()
        C_behind = np.zeros_like(C)
        Tb = np.ones_like(T)
        for k in range(rank + 1, world):
            C_behind = C_behind + Tb[..., None] * gathered[k][..., :3].numpy()
            Tb = Tb * gathered[k][..., 3].numpy()
        g_slab = T_front[..., None] * g
        gr = oracle.backward(mine, cam, g_slab, opts)
        w = np.zeros_like(g)
        w[..., 0] = (g_slab * C_behind).sum(axis=-1)
        gw = oracle.backward(_white(mine), cam, w, opts)
        out = {}
        for k in ("means", "scales", "quats", "opacities", "sh"):
            out[k] = gr[k] - (gw[k] if k != "sh" else 0.0)
        np.savez(os.path.join(out_dir, f"slab_{rank}.npz"), ids=ids, C=C, T=T, **out)
    finally:
        dist.destroy_process_group()


def test_depth_slab_compositing_matches_full_render(tmp_path):
    _spawn(_slab_worker, str(tmp_path))
    scene, cam, g = _slab_scene()
    opts = oracle.opts_array(t_cull=0.0)
    full = oracle.render(scene, cam, opts)
    fb = oracle.backward(scene, cam, g, opts)
    parts = [np.load(tmp_path / f"slab_{r}.npz") for r in range(WORLD)]
    assert all(p["ids"].size > 0 for p in parts)
    for p in parts:                                  # every rank composites the same image
        np.testing.assert_allclose(p["C"], full["color"], rtol=0, atol=1e-12)
        np.testing.assert_allclose(p["T"], full["T"], rtol=0, atol=1e-12)
    assert full["color"].max() > 0.1                 # the view is not empty
    for k in ("means", "scales", "quats", "opacities", "sh"):
        got = np.zeros_like(fb[k])
        for p in parts:
            got[p["ids"]] = p[k]
        ref = fb[k]
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-30)
        assert err < 1e-6, (k, err)
