#!/usr/bin/env python
"""Benchmark: forward + backward of one view of a 3.0M-splat scene at 1256x828.

A step is one pass of the whole path over one view: projection, depth sort,
binning, forward blending, summed L1 loss, backward blending with per-splat
reduction, and the chain rule to the 3D parameters.  Inputs are resident in
HBM; the scene's parameters (708 MB) are larger than L2.  One JSON line on
stdout (rank 0).

  python bench.py [--gpus N --steps K --warmup W]         the CUDA path
  python bench.py --impl reference [...]                  the FP64 CPU oracle

Under torchrun each rank renders its own view of the same scene (orbit angle
2 pi rank / N): views are independent, so no data-path collective (weak
scaling); ranks only meet at barriers and for the max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd ms/view, splat-frags/s at 3M/1256x828, FP16 vs FP32 state; p99 latency"
WORKLOAD = "mipnerf360-shaped synthetic scene, 3.0M splats SH3, 1256x828, L1 loss, fwd+bwd"
N_SPLATS = 3_000_000
STAGES = ("project", "sort", "bin", "blend_fwd", "loss", "blend_bwd", "project_bwd")
KERNELS_PER_STAGE = {"project": 1, "sort": 5, "bin": None, "blend_fwd": 1, "loss": 1,
                     "blend_bwd": 2, "project_bwd": 1}   # bin: 2 + pair-sort passes
# Nominal FP32 rate (SM count x FP32 lanes x 2 flop x max SM clock): raster stages are
# plain FP32 ALU work, for which the measured peaks carry no figure.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
FLOP_PER_FRAG_FWD = 20.0
FLOP_PER_FRAG_BWD = 70.0
REF_PIXELS = 64    # pixels traced per step of the reference (oracle) arm


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=N_SPLATS, help="splat count (smaller for profiling)")
    ap.add_argument("--no-extras", action="store_true",
                    help="main timed loop only (no fp16 run, e2e, CPU baseline, clocks)")
    ap.add_argument("--cpu-pixels", type=int, default=768, help="pixels in the CPU-baseline sample")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-stream measurement")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--no-training", action="store_true", help="skip the training-step measurement")
    ap.add_argument("--ablation-only", action="store_true",
                    help="only the gradient-reduction ablation (one backward raster per mode after "
                         "a warm-up; for counting atomics under a profiler)")
    return ap.parse_args()


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the CUDA path
# ---------------------------------------------------------------------------
def replica_orbit_angle(rank: int, world: int) -> float:
    """Each rank renders its own view: orbit angle 2 pi rank / world."""
    return 2.0 * math.pi * rank / world


def max_over_ranks_ms(total_ms: float, device, world: int) -> float:
    """Elapsed time of the job: the slowest rank's (MAX all-reduce; a no-op at N = 1)."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    if world > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world, local_rank):
    import torch
    import paper_2505_18764_gb300 as gs
    from paper_2505_18764_gb300 import _lib
    import synthetic as syn

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    t0 = time.time()
    scene_np, cam0, target_np = syn.mipnerf_scene_3m(args.n)
    cam = syn.orbit_camera(replica_orbit_angle(rank, world), 4.0, 50.0, cam0.width, cam0.height)
    log(f"[rank {rank}] scene generated in {time.time() - t0:.1f}s")
    scene = gs.SceneTensors.from_numpy(scene_np, dev)
    target = torch.from_numpy(target_np).to(dev)
    H, W = cam.height, cam.width
    opts = gs.RasterOpts(state_format="fp32", sh_degree=3, t_cull=1e-4)
    ws = gs.Workspace(scene.n, W, H, opts, device=dev)
    ccam = gs.camera_to_c(cam)
    stream = torch.cuda.current_stream(dev)
    image = torch.empty((H, W, 3), dtype=torch.float32, device=dev)
    last = torch.empty((H, W), dtype=torch.int32, device=dev)
    dl = torch.empty_like(image)
    loss = torch.empty(1, dtype=torch.float64, device=dev)
    grads = gs.zero_grads(scene)

    def make_step(ws, o, state):
        def step(events=None):
            def mark(i):
                if events is not None:
                    events[i].record(stream)
            mark(0)
            gs.project(ws, scene, ccam, o, stream)
            mark(1)
            gs.sort(ws, stream)
            mark(2)
            gs.bin(ws, ccam, o, stream)
            mark(3)
            gs.blend_forward(ws, ccam, o, image, state, last, None, stream)
            mark(4)
            gs.loss(image, target, "l1", dl, loss, stream)
            mark(5)
            gs.blend_backward(ws, ccam, o, state, last, dl, stream)
            mark(6)
            gs.project_backward(ws, scene, ccam, o, grads, stream)
            mark(7)
        return step

    def timed(step, K, W_):
        for _ in range(W_):
            step()
        torch.cuda.synchronize(dev)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(8)] for _ in range(K)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter()
        for k in range(K):
            step(ev[k])
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        total = ev[0][0].elapsed_time(ev[-1][7])
        per = {s: float(np.mean([ev[k][i].elapsed_time(ev[k][i + 1]) for k in range(K)]))
               for i, s in enumerate(STAGES)}
        step_ms = [ev[k][0].elapsed_time(ev[k][7]) for k in range(K)]
        return total, per, step_ms, t_wall

    state32 = gs.alloc_state(H, W, "fp32", dev)
    step32 = make_step(ws, opts, state32)
    clocks = ClockSampler(local_rank)
    # warm-up, then the timed region for the headline number
    for _ in range(args.warmup):
        step32()
    torch.cuda.synchronize(dev)
    if args.ablation_only:
        return dict(metric=METRIC, reduction_ablation=run_ablation(gs, torch, ws, ccam, state32, last,
                                                                   dl, stream, None, reps=1))
    # stage times: the same step as separate calls, events between the stages
    eager_ms, per_stage, _, _ = timed(step32, args.steps, 0)

    # the headline: each view as one gs_render_batch_graph call (the step's
    # launches captured into a CUDA graph, updated in place from view to view)
    gstream = torch.cuda.Stream(dev)
    gout = dict(image=image, state=state32, last=last, dL_dimage=dl, loss=loss, grads=grads)

    def graph_step():
        gs.render_batch([gs.Request(scene, ccam, opts, backward=True, loss_kind="l1",
                                    target=target, outputs=gout)], ws, gstream, graph=True)

    def timed_graph(K, W_):
        gstream.wait_stream(stream)
        with torch.cuda.stream(gstream):
            for _ in range(W_):
                graph_step()
        torch.cuda.synchronize(dev)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(K)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter()
        with torch.cuda.stream(gstream):
            for k in range(K):
                ev[k][0].record(gstream)
                graph_step()
                ev[k][1].record(gstream)
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall
        return (ev[0][0].elapsed_time(ev[-1][1]), [e[0].elapsed_time(e[1]) for e in ev], t_wall)

    if not args.no_extras:
        clocks.start()
    total_ms, step_ms, t_wall = timed_graph(args.steps, max(args.warmup, 2))
    clk = clocks.stop() if not args.no_extras else None
    gs.check_status(ws, stream)
    total_ms_max = max_over_ranks_ms(total_ms, dev, world)
    ms_per_view = total_ms_max / (args.steps * world)

    # counters of this view (untimed): visible splats, pairs, fragments
    out = gs.render(ws, scene, ccam, opts, stream, want_n_contrib=True)
    cnt = gs.read_counters(ws, stream)
    F = int(out["n_contrib"].sum().item())
    n_front = int(((scene.means @ torch.as_tensor(cam.viewmat[2, :3], device=dev)) +
                   float(cam.viewmat[2, 3]) > 0.2).sum().item())
    V, P = cnt["visible"], cnt["pairs"]
    P_live = cnt["live_pairs"]
    npix = H * W
    passes = ws.c.pair_passes
    # project; sort: setup (epoch, tile counters) + 4 passes; bin: count, chunk setup, emit,
    # pair-sort passes, ranges, item order; blend_fwd; loss; blend_bwd: item reorder +
    # raster; project_bwd
    kernels_per_step = 1 + 5 + (3 + passes + 2) + 1 + 1 + 2 + 1
    K_sh = 16

    # algorithmic bytes (HBM-bound stages) and flops (raster stages) per launch
    alg = {
        "project": ("hbm", scene.n * 20 + n_front * 28 + V * (12 * K_sh + 48)),
        "sort": ("hbm", scene.n * 4 + 56 * V),
        # emission writes P pairs, the first pass reads them and writes the live
        # ones, later passes move live pairs, the ranges kernel reads them
        "bin": ("hbm", 148 * V + 16 * P + (8 + 16 * (passes - 1) + 4) * P_live),
        "blend_fwd": ("alu", FLOP_PER_FRAG_FWD * F),
        "loss": ("hbm", 36 * npix),
        "blend_bwd": ("alu", FLOP_PER_FRAG_BWD * F),
        "project_bwd": ("hbm", V * (48 + 236 + 2 * 236)),
    }
    # the FP32 FMA rate measured on this GPU, reported beside the derived peak
    fma_tflops = gs.fp32_fma_rate(1 << 16, stream)
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    stage_roof = {}
    for s, (bound, amount) in alg.items():
        ms = per_stage[s]
        if bound == "hbm":
            ach = amount / (ms * 1e-3) / 1e9
            stage_roof[s] = dict(bound="hbm", achieved=round(ach, 1), unit="GB/s",
                                 frac=round(ach / hbm_peak, 4), ms=round(ms, 4))
        else:
            ach = amount / (ms * 1e-3) / 1e12
            stage_roof[s] = dict(bound="alu", achieved=round(ach, 3), unit="TFLOP/s",
                                 frac=round(ach / FP32_PEAK_TFLOPS, 4),
                                 frac_of_measured_fma=round(ach / fma_tflops, 4), ms=round(ms, 4))
    # step bound: each stage at its own roofline (bytes / measured HBM peak, or
    # flops / FP32 peak), summed over the stages; the step's fraction of it
    bound_ms = {s: (amount / (hbm_peak * 1e9) if bound == "hbm"
                    else amount / (FP32_PEAK_TFLOPS * 1e12)) * 1e3
                for s, (bound, amount) in alg.items()}
    step_bound = dict(ms=round(sum(bound_ms.values()), 4),
                      stages_ms={s: round(v, 4) for s, v in bound_ms.items()},
                      note="sum over stages of max(bytes / HBM peak, flops / FP32 peak) with each "
                           "stage's algorithmic amount (one bound applies per stage)")
    dom = max(per_stage, key=per_stage.get)
    dr = stage_roof[dom]
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        tj = json.load(open(tfile))
        if tj.get("kernel_stage") == dom and \
                tj.get("source_hash") == _source_hash(tj.get("source_files", [])):
            traffic = tj.get("bytes_per_launch")
    roofline = dict(kernel=dom, bound=dr["bound"], achieved=dr["achieved"],
                    peak=round(hbm_peak, 1) if dr["bound"] == "hbm" else round(FP32_PEAK_TFLOPS, 2),
                    unit=dr["unit"], frac=dr["frac"], traffic=traffic,
                    peak_source="MEASURED_PEAKS.json hbm_gbs (measured)" if dr["bound"] == "hbm"
                    else "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz (derived)")
    if dr["bound"] == "alu":
        roofline.update(peak_measured_fma=round(fma_tflops, 2),
                        frac_of_measured_fma=round(dr["achieved"] / fma_tflops, 4))

    res = dict(metric=METRIC, value=round(ms_per_view, 4), unit="ms/view", n_gpus=world,
               steps=args.steps, warmup=args.warmup, ms_per_step=round(total_ms_max / args.steps, 4),
               higher_is_better=False, scaling="weak", vs_baseline=None, dtype="f32",
               data="synthetic",
               config=dict(workload=WORKLOAD, splats=scene.n, width=W, height=H, sh_degree=3,
                           state_format="fp32", t_cull=1e-4, reduce="warp", loss="l1",
                           views_per_step=world, parallelism=f"replicas x{world}",
                           l2="inputs larger than L2 (scene parameters 708 MB > 129 MB)"),
               counts=dict(visible=V, pairs=P, live_pairs=P_live, fragments=F, in_front=n_front,
                           pixels=npix),
               splat_frags_per_s=round(F / (ms_per_view * 1e-3), 1),
               schedule="one gs_render_batch_graph call per view (the step as one CUDA graph)",
               eager_ms_per_view=round(eager_ms / args.steps, 4),
               stages_ms=per_stage, stage_roofline=stage_roof,
               p50_ms=round(float(np.percentile(step_ms, 50)), 4),
               p99_ms=round(float(np.percentile(step_ms, 99)), 4),
               wall_ms_per_step=round(t_wall * 1e3 / args.steps, 4),
               gpu_launches=kernels_per_step * args.steps * world,
               roofline=roofline, step_bound=step_bound)

    step_bound["frac_of_step"] = round(step_bound["ms"] / ms_per_view, 4)
    if not args.no_extras:
        # FP16 saved state, same work otherwise
        o16 = gs.RasterOpts(state_format="fp16", sh_degree=3, t_cull=1e-4)
        ws16 = gs.Workspace(scene.n, W, H, o16, device=dev)
        st16 = gs.alloc_state(H, W, "fp16", dev)
        tot16, per16, _, _ = timed(make_step(ws16, o16, st16), args.steps, args.warmup)
        res["fp16_state"] = dict(ms_per_view=round(tot16 / args.steps, 4),
                                 speedup_vs_fp32=round((eager_ms / args.steps) / (tot16 / args.steps), 4),
                                 stages_ms=per16)
        del ws16
        res["e2e"] = run_e2e(args, gs, torch, scene, target, ccam, opts, dev, stream, image, state32,
                             last, dl, loss, grads, ws)
        res["reduction_ablation"] = run_ablation(gs, torch, ws, ccam, state32, last, dl, stream, F)
        res["back_to_front"] = run_backward_order(gs, torch, ws, ccam, state32, last, dl, stream)
        res["memory_efficiency"] = run_chunked(args, gs, torch, scene, ccam, target, dev, stream)
        if not args.no_training:
            res["training"] = run_training(args, dev)
        res["clocks"] = clk
        if not args.no_serving:
            res["serving"] = run_serving(args, dev)
        if world == 1:
            res["cpu_baseline"] = cpu_baseline(args, scene_np, cam, target_np)
    return res


# Gradient reduction modes of the backward raster (the paper's Sec. 3.2 ablation):
# per-fragment atomics, and the warp reduction with balancing thresholds X.
ABLATION = (("fragment", 0), ("naive", 0), ("warp", 1), ("warp", 4), ("warp", 8), ("warp", 16), ("warp", 33))


def run_ablation(gs, torch, ws, ccam, state, last, dl, stream, F, reps=10):
    """Backward-raster time per reduction mode on the view the workspace holds
    (binning, state and dL/dC from the last step)."""
    out = []
    for mode, x in ABLATION:
        o = gs.RasterOpts(state_format="fp32", sh_degree=3, t_cull=1e-4, reduce_mode=mode,
                          reduce_threshold=x)
        gs.blend_backward(ws, ccam, o, state, last, dl, stream)   # warm-up
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        for k in range(reps):
            ev[2 * k].record(stream)
            gs.blend_backward(ws, ccam, o, state, last, dl, stream)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.median([ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(reps)]))
        row = dict(mode=mode, X=x, blend_bwd_ms=round(ms, 4))
        if F:
            row["splat_frags_per_s"] = round(F / (ms * 1e-3), 1)
        out.append(row)
    return out


def run_backward_order(gs, torch, ws, ccam, state, last, dl, stream, reps=10):
    """Backward-raster time front to back (the default) and back to front (T
    recovered by division from the stored final transmittance)."""
    out = {}
    for order in ("front_to_back", "back_to_front"):
        o = gs.RasterOpts(state_format="fp32", sh_degree=3, t_cull=1e-4, backward_order=order)
        gs.blend_backward(ws, ccam, o, state, last, dl, stream)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * reps)]
        for k in range(reps):
            ev[2 * k].record(stream)
            gs.blend_backward(ws, ccam, o, state, last, dl, stream)
            ev[2 * k + 1].record(stream)
        torch.cuda.synchronize()
        out[order + "_ms"] = round(float(np.median([ev[2 * k].elapsed_time(ev[2 * k + 1])
                                                    for k in range(reps)])), 4)
    return out


def run_chunked(args, gs, torch, scene, ccam, target, dev, stream, caps=(1 << 20, 1 << 18)):
    """The same view in the memory-efficiency mode: a small fixed pair capacity,
    the depth order binned and rasterized in chunks that fit it.  Reports time
    per view (fwd + bwd through gs_raster_forward / gs_raster_backward), chunk
    count and workspace bytes against the default single-pass workspace."""
    W, H = ccam.width, ccam.height
    o_def = gs.RasterOpts(state_format="fp32", sh_degree=3, t_cull=1e-4)
    ws_def = gs.Workspace(scene.n, W, H, o_def, device=dev)
    sb = ws_def.sort_bytes()
    out = dict(default_workspace_bytes=gs.Workspace.required_bytes(scene.n, W, H, o_def),
               default_pair_capacity=max(16 * scene.n, 1 << 22),
               default_sort_bytes=sb["depth_sort"] + sb["pair_sort"],
               default_sort_bytes_split=sb, runs=[])
    del ws_def
    grads = gs.zero_grads(scene)
    for cap in caps:
        o = gs.RasterOpts(state_format="fp32", sh_degree=3, t_cull=1e-4, chunked=True,
                          pair_capacity=cap)
        ws = gs.Workspace(scene.n, W, H, o, device=dev)
        image = torch.empty((H, W, 3), device=dev)
        state = gs.alloc_state(H, W, "fp32", dev)
        last = torch.empty((H, W), dtype=torch.int32, device=dev)
        dl = torch.empty((H, W, 3), device=dev)
        loss = torch.zeros(1, dtype=torch.float64, device=dev)

        def step():
            gs.project(ws, scene, ccam, o, stream)
            gs.sort(ws, stream)
            gs.raster_forward(ws, ccam, o, image, state, last, None, stream=stream)
            gs.loss(image, target, "l1", dl, loss, stream)
            gs.raster_backward(ws, scene, ccam, o, state, last, dl, grads, stream)

        step()
        torch.cuda.synchronize(dev)
        K = 5
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        gs.check_status(ws, stream)
        sb = ws.sort_bytes()
        out["runs"].append(dict(pair_capacity=cap, chunks=int(ws.c.n_chunks),
                                workspace_bytes=int(ws.nbytes),
                                sort_bytes=sb["depth_sort"] + sb["pair_sort"], sort_bytes_split=sb,
                                pair_buffer_bytes=4 * 4 * cap,
                                ms_per_view=round(a.elapsed_time(b) / K, 4)))
        del ws
    return out


def run_training(args, dev):
    """Training step through torch.autograd: 1.0M splats (tiny-scene
    distributions, SH3), 8 orbit views at 1600x1060, FP16 state, summed L2
    loss per view, then an Adam step (lr 1e-3) on every parameter."""
    import torch
    import synthetic as syn
    from paper_2505_18764_gb300 import RasterOpts
    from paper_2505_18764_gb300.autograd import Renderer
    scene_np, cams, targets = syn.training_scene_1m()
    model = Renderer(scene_np, 1600, 1060, RasterOpts(state_format="fp16", sh_degree=3),
                     device=dev)
    tg = [torch.from_numpy(t).to(dev) for t in targets]
    optim = torch.optim.Adam(model.parameters(), lr=1e-3)

    def step():
        optim.zero_grad(set_to_none=False)
        total = torch.zeros((), dtype=torch.float32, device=dev)
        for cam, t in zip(cams, tg):
            loss = ((model(cam) - t) ** 2).sum()
            loss.backward()
            total += loss.detach()
        optim.step()
        return total

    for _ in range(2):
        step()
    torch.cuda.synchronize(dev)
    K = 5
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record()
    losses = []
    for k in range(K):
        losses.append(step())
        ev[k + 1].record()
    torch.cuda.synchronize(dev)
    ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(K)]
    return dict(config="1.0M splats SH3, 8 views 1600x1060, fp16 state, summed L2, Adam lr 1e-3",
                ms_per_step=round(float(np.median(ms)), 3),
                ms_per_view=round(float(np.median(ms)) / len(cams), 3),
                loss_first=round(float(losses[0].item()), 1), loss_last=round(float(losses[-1].item()), 1),
                steps=K)


def run_e2e(args, gs, torch, scene, target, ccam, opts, dev, stream, image, state, last, dl, loss,
            grads, ws):
    """The step through the C ABI with host buffers.  The scene's parameters are
    model state and stay resident (as in training and serving); every step
    copies its inputs, the camera and the target image, from pinned host memory
    and reads its result, the loss, back.  `stateless` also copies the whole
    scene up and every gradient down each step."""
    host_tgt = target.cpu().pin_memory()
    host_loss = loss.cpu().pin_memory()
    gnames = ("means", "scales", "quats", "opacities", "sh")

    def step_resident(k=0):
        target.copy_(host_tgt, non_blocking=True)   # the camera travels by value in the call
        for g in gnames:
            grads[g].zero_()
        gs.project(ws, scene, ccam, opts, stream)
        gs.sort(ws, stream)
        gs.raster_forward(ws, ccam, opts, image, state, last, None, stream=stream)
        gs.loss(image, target, "l1", dl, loss, stream)
        gs.raster_backward(ws, scene, ccam, opts, state, last, dl, grads, stream)
        host_loss.copy_(loss, non_blocking=True)

    # The same step scheduled as a training loop would: step k+1's target is
    # copied up on a copy stream into the other of two buffers while step k
    # computes, and the gradient arrays hold this view's gradients alone without
    # zeroing all n rows: the backward projection stores the visible splats'
    # rows (zero_touched = 2) and the rows of splats that left the view are
    # zeroed.  Every step still copies its own target up and reads its loss back
    # (into pinned host memory, inside the graph) in the timed region.  The step
    # is one gs_render_batch_graph call (a CUDA graph) on its own stream.
    st = torch.cuda.Stream(dev)
    copy_st = torch.cuda.Stream(dev)
    tgt_buf = [target, torch.empty_like(target)]
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    gout = dict(image=image, state=state, last=last, dL_dimage=dl, loss=loss, grads=grads)

    def issue_copy(k):
        copy_st.wait_stream(st)   # the buffer's previous reader (step k - 2's loss) is done
        with torch.cuda.stream(copy_st):
            tgt_buf[k % 2].copy_(host_tgt, non_blocking=True)
        copied[k % 2].record(copy_st)

    def step_pipelined(k, last_k):
        if k + 1 <= last_k:
            issue_copy(k + 1)
        st.wait_event(copied[k % 2])
        # one graph: zero the previous view's gradient rows, the step, the loss to the host
        gs.render_batch([gs.Request(scene, ccam, opts, backward=True, loss_kind="l1",
                                    target=tgt_buf[k % 2], outputs=gout, zero_touched=2,
                                    loss_host=host_loss)], ws, st, graph=True)

    def timed_pipelined():
        st.wait_stream(stream)
        with torch.cuda.stream(st):
            for g in gnames:
                grads[g].zero_()
        issue_copy(0)
        W_ = max(args.warmup, 2)
        for k in range(W_):
            step_pipelined(k, W_ - 1)
        torch.cuda.synchronize(dev)
        K = max(1, min(args.steps, 20))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        issue_copy(0)
        for k in range(K):
            step_pipelined(k, K - 1)
        b.record(st)
        torch.cuda.synchronize(dev)
        return round(a.elapsed_time(b) / K, 4), K

    host_in = [t.cpu().pin_memory() for t in scene.tensors()] + [host_tgt]
    dev_in = list(scene.tensors()) + [target]
    host_out = [grads[k].cpu().pin_memory() for k in gnames] + [host_loss]
    dev_out = [grads[k] for k in gnames] + [loss]

    def step_stateless():
        for h, d in zip(host_in, dev_in):
            d.copy_(h, non_blocking=True)
        for g in gnames:
            grads[g].zero_()
        gs.project(ws, scene, ccam, opts, stream)
        gs.sort(ws, stream)
        gs.raster_forward(ws, ccam, opts, image, state, last, None, stream=stream)
        gs.loss(image, target, "l1", dl, loss, stream)
        gs.raster_backward(ws, scene, ccam, opts, state, last, dl, grads, stream)
        for h, d in zip(host_out, dev_out):
            h.copy_(d, non_blocking=True)

    def timed_steps(step):
        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize(dev)
        K = max(1, min(args.steps, 20))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            step()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return round(a.elapsed_time(b) / K, 4), K

    v, K = timed_pipelined()
    v1, _ = timed_steps(step_resident)
    v2, _ = timed_steps(step_stateless)
    return dict(value=v, unit="ms/view",
                h2d_bytes_per_step=host_tgt.numel() * host_tgt.element_size(),
                d2h_bytes_per_step=host_loss.numel() * host_loss.element_size(), steps=K,
                inputs="target image up, loss down; scene parameters resident",
                schedule="one gs_render_batch_graph call per step; next target copied up "
                         "during the step; gradient rows stored for the visible splats and "
                         "zeroed for those that left the view (zero_touched = 2); loss copied "
                         "to pinned host memory in the graph",
                serial=dict(value=v1, unit="ms/view",
                            schedule="copy up, zero all gradient rows, step, loss down, in one "
                                     "stream"),
                stateless=dict(value=v2, unit="ms/view",
                               h2d_bytes_per_step=sum(t.numel() * t.element_size() for t in host_in),
                               d2h_bytes_per_step=sum(t.numel() * t.element_size() for t in host_out)))


def run_serving(args, dev):
    """Serving stream: Poisson arrivals at 200/s over four resident scenes
    (0.5M, 1.5M, 3M, 6M splats, tiny-scene distributions, SH3), resolutions
    drawn from 640x360 .. 3840x2160, 80% renders and 20% fine-tune steps,
    admitted under a 120 GB HBM budget, FP16 state."""
    import paper_2505_18764_gb300 as gs
    from paper_2505_18764_gb300.serving import CudaExecutor, Server, make_requests
    import synthetic as syn
    t0 = time.time()
    scenes = [gs.SceneTensors.from_numpy(syn.cube_scene(n, seed=50 + i, sh_degree=3), dev)
              for i, n in enumerate(syn.SERVING_SCENE_SIZES)]
    log(f"serving scenes ready in {time.time() - t0:.1f}s")
    specs = syn.serving_requests(args.serve_requests, 200.0, seed=5)

    def cam_for(s):
        return syn.orbit_camera(s["angle"], 4.0, 60.0, s["width"], s["height"])

    ex = CudaExecutor(scenes, n_slots=8, reuse_outputs=True)
    # warm-up (untimed): every (scene, resolution, mode) once, which also sizes
    # the pair capacity of each combination
    combos = [dict(arrival=0.0, scene=si, width=w, height=h, backward=b, angle=0.3 * si + 0.1 * ri)
              for si in range(len(scenes)) for ri, (w, h) in enumerate(syn.SERVING_RESOLUTIONS)
              for b in (False, True)]
    warm = make_requests(combos, cam_for)
    Server(ex, hbm_budget_bytes=120 << 30, max_slots=8).run(warm, realtime=False, keep_results=False)
    reqs = make_requests(specs, cam_for)
    srv = Server(ex, hbm_budget_bytes=120 << 30, max_slots=8)
    ex.gpu_ms.clear()
    stats = srv.run(reqs, realtime=True, keep_results=False)
    stats["gpu_ms_per_request_mean"] = float(np.mean(ex.gpu_ms)) if ex.gpu_ms else None
    # sum of the requests' device spans over the wall time (streams overlap, so
    # above 1 means several requests were on the GPU at once)
    stats["device_span_share"] = float(np.sum(ex.gpu_ms) / (stats["wall_s"] * 1e3))
    fwd = [r.latency for r in reqs if r.status == "done" and not r.backward]
    bwd = [r.latency for r in reqs if r.status == "done" and r.backward]
    stats["p99_fwd_ms"] = float(np.percentile(fwd, 99) * 1e3) if fwd else None
    stats["p99_fwdbwd_ms"] = float(np.percentile(bwd, 99) * 1e3) if bwd else None
    stats["config"] = ("2000 Poisson arrivals at 200/s, scenes 0.5M/1.5M/3M/6M splats SH3, "
                       "640x360..3840x2160, 20% fwd+bwd, 120 GB budget, fp16 state, 8 slots")
    return {k: (round(v, 3) if isinstance(v, float) else v) for k, v in stats.items()}


def _source_hash(files):
    """Hash of the kernel sources the stored DRAM counters were taken from:
    the counters stand only while those files are unchanged."""
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2505_18764_gb300", "csrc")
    for f in sorted(files):
        p = os.path.join(d, f)
        if not os.path.exists(p):
            return None
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16] if files else None


# ---------------------------------------------------------------------------
# the FP64 CPU oracle
# ---------------------------------------------------------------------------
def oracle_sample(scene_np, cam, target_np, n_pixels, seed):
    """One bounded sample of the view: full preprocessing (projection + depth
    order of every splat), the forward of n_pixels random pixels, the true
    L1 gradient sign(C - target) there, and their backward; the tracing time
    is extrapolated to the whole image (preprocessing counted once)."""
    import oracle
    rng = np.random.default_rng(seed)
    pix = rng.choice(cam.width * cam.height, size=n_pixels, replace=False).astype(np.int32)
    opts = oracle.opts_array(t_cull=1e-4)
    t0 = time.perf_counter()
    fwd = oracle.render(scene_np, cam, opts, pixels=pix, timings=True)
    g = np.zeros((cam.height * cam.width, 3))
    g[pix] = np.sign(fwd["color"] - target_np.reshape(-1, 3)[pix].astype(np.float64))
    out = oracle.backward(scene_np, cam, g, opts, pixels=pix, timings=True)
    wall = time.perf_counter() - t0
    tf, tb = fwd["timings"], out["timings"]
    trace = tf["trace_s"] + tb["trace_s"]
    tm = dict(preprocess_s=tb["preprocess_s"], trace_s=trace)
    est_s = tm["preprocess_s"] + trace * (cam.width * cam.height) / n_pixels
    return est_s, wall, tm


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(args, scene_np, cam, target_np):
    import oracle
    import synthetic as syn
    est_s, wall, tm = oracle_sample(scene_np, cam, target_np, args.cpu_pixels, seed=123)
    # the tiny scene (1,024 splats, 128x128, L2 loss) in full, on one core
    tiny, tcam, ttgt = syn.tiny_scene_1k()
    cores = oracle.num_threads()
    oracle.set_threads(1)
    t0 = time.perf_counter()
    img = oracle.render(tiny, tcam)["color"]
    oracle.backward(tiny, tcam, 2.0 * (img - ttgt.astype(np.float64)))
    tiny_s = time.perf_counter() - t0
    oracle.set_threads(0)
    return dict(value=round(est_s * 1e3, 1), unit="ms/view", cores=cores,
                cpu_model=cpu_model(), kind="oracle",
                tiny_scene_single_thread_ms=round(tiny_s * 1e3, 1),
                sample=(f"FP64 oracle: projection + depth order of all {scene_np.n} splats "
                        f"({tm['preprocess_s']:.2f}s), then forward, true L1 gradient and backward "
                        f"of {args.cpu_pixels} random pixels ({tm['trace_s']:.2f}s), trace time "
                        f"scaled by {cam.width * cam.height}/{args.cpu_pixels} pixels; "
                        f"wall {wall:.1f}s"))


def run_reference(args, rank, world):
    import oracle
    import synthetic as syn
    if rank != 0:
        return None
    scene_np, cam, target_np = syn.mipnerf_scene_3m(args.n)
    oracle.build()
    for w in range(args.warmup):
        oracle_sample(scene_np, cam, target_np, 16, seed=w)
    ests, walls = [], []
    # each step a bounded sample: REF_PIXELS pixels keep the whole --steps run
    # within minutes (about a second per step on 16 cores)
    for k in range(args.steps):
        est_s, wall, _ = oracle_sample(scene_np, cam, target_np, REF_PIXELS, seed=1000 + k)
        ests.append(est_s)
        walls.append(wall)
    v = float(np.mean(ests)) * 1e3
    return dict(metric=METRIC, value=round(v, 1), unit="ms/view", n_gpus=world, steps=args.steps,
                warmup=args.warmup, ms_per_step=round(v, 1), higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=WORKLOAD, splats=scene_np.n, width=cam.width,
                            height=cam.height, sh_degree=3, state_format="fp64 (no rounding)",
                            t_cull=1e-4, loss="l1"),
                cpu_baseline=dict(value=round(v, 1), unit="ms/view", cores=oracle.num_threads(),
                                  kind="oracle",
                                  sample=f"per step: all-splat preprocessing + forward, true L1 "
                                         f"gradient and backward of {REF_PIXELS} random "
                                         f"pixels, trace time scaled to the full view"),
                e2e=dict(value=round(v, 1), unit="ms/view", h2d_bytes_per_step=0,
                         d2h_bytes_per_step=0),
                wall_s_per_step=round(float(np.mean(walls)), 2))


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
