"""Continuous-batching render server.

Scenes stay resident on the device.  Requests (a novel-view render, or a
forward + backward fine-tune step that returns the loss and the per-splat
gradients without changing the resident scene) arrive over time.  The
scheduler admits the oldest waiting request as soon as a slot is free and its
device memory (workspace + outputs, computed exactly from gs_workspace_size)
fits under the HBM budget; admitted requests run on their slot's own CUDA
stream, so work that arrives while others are on the GPU overlaps with them.
Latency = completion - arrival; the server reports p50 / p99 latency and
views per second.

Execution is behind a small executor interface (memory / submit / poll /
finish), so the scheduling, admission, cancellation and failure handling run
unchanged against a host-only fake in tests.
"""
from __future__ import annotations

import collections
import ctypes
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass
class ServeRequest:
    rid: int
    scene: int                   # index into the server's resident scenes
    camera: object               # width, height, viewmat, ... (see camera_to_c)
    backward: bool = False       # fine-tune step: L2 loss against `target`, gradients returned
    arrival: float = 0.0         # seconds after the run starts
    target_seed: int = 0         # the fine-tune target image is drawn from this seed
    # filled in by the server
    t_admit: float | None = None
    t_done: float | None = None
    status: str = "pending"      # pending | waiting | running | done | failed | cancelled | rejected
    error: str | None = None
    retries: int = 0
    result: dict = field(default_factory=dict)

    @property
    def latency(self):
        return None if self.t_done is None else self.t_done - self.arrival


class Retry(Exception):
    """Raised by an executor's finish() when a request must run again (for
    example with a larger pair capacity); the request keeps its arrival time."""


class Server:
    def __init__(self, executor, hbm_budget_bytes: int, max_slots: int = 8):
        self.ex = executor
        self.budget = int(hbm_budget_bytes)
        self.max_slots = int(max_slots)
        self.in_flight_bytes = 0
        self.peak_bytes = 0
        self.peak_concurrency = 0
        self._cancelled = set()

    def cancel(self, rid: int):
        """Withdraw a request that has not been admitted yet."""
        self._cancelled.add(rid)

    def run(self, requests, realtime: bool = True, idle_sleep: float = 1e-4,
            keep_results: bool = True):
        """Serve `requests` (arrival times relative to the start); returns stats.
        With keep_results=False a request's outputs are dropped when it
        completes (only scalars such as the loss are kept), as a server that
        has delivered its responses would."""
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        waiting = collections.deque()
        running = []          # (request, handle, bytes)
        free_slots = list(range(self.max_slots))
        t0 = time.perf_counter()
        now = 0.0
        while pending or waiting or running:
            now = time.perf_counter() - t0
            if not realtime:  # simulated clock: jump to the next arrival when idle
                if not waiting and not running and pending:
                    now = max(now, pending[0].arrival)
            while pending and (pending[0].arrival <= now or not realtime):
                r = pending.popleft()
                r.status = "waiting"
                waiting.append(r)
            progressed = False
            # completions
            still = []
            for r, h, nbytes in running:
                if self.ex.poll(h):
                    self.in_flight_bytes -= nbytes
                    free_slots.append(h.slot)
                    progressed = True
                    try:
                        res = self.ex.finish(h)
                        r.result = res if keep_results else {
                            k: v for k, v in res.items() if isinstance(v, (int, float))}
                        r.status = "done"
                    except Retry:
                        r.status = "waiting"
                        r.retries += 1
                        waiting.appendleft(r)
                        continue
                    except Exception as e:  # a failed request does not stop the server
                        r.status, r.error = "failed", str(e)
                    r.t_done = time.perf_counter() - t0
                else:
                    still.append((r, h, nbytes))
            running = still
            # admissions, oldest first; a request that can never fit is rejected
            while waiting and free_slots:
                r = waiting[0]
                if r.rid in self._cancelled:
                    waiting.popleft()
                    r.status = "cancelled"
                    progressed = True
                    continue
                need = self.ex.memory(r)
                if need > self.budget:
                    waiting.popleft()
                    r.status, r.error = "rejected", f"needs {need} B, budget {self.budget} B"
                    progressed = True
                    continue
                if self.in_flight_bytes + need > self.budget:
                    break  # wait for memory to free up
                waiting.popleft()
                slot = free_slots.pop()
                r.t_admit = time.perf_counter() - t0
                r.status = "running"
                try:
                    h = self.ex.submit(r, slot)
                except Exception as e:
                    r.status, r.error = "failed", str(e)
                    r.t_done = time.perf_counter() - t0
                    free_slots.append(slot)
                    progressed = True
                    continue
                self.in_flight_bytes += need
                self.peak_bytes = max(self.peak_bytes, self.in_flight_bytes)
                running.append((r, h, need))
                self.peak_concurrency = max(self.peak_concurrency, len(running))
                progressed = True
            if not progressed:
                if realtime and not waiting and not running and pending:
                    time.sleep(max(0.0, min(pending[0].arrival - now, 0.005)))
                else:
                    time.sleep(idle_sleep)
        return self.stats(requests, time.perf_counter() - t0)

    def stats(self, requests, wall):
        lat = np.array([r.latency for r in requests if r.status == "done"], dtype=np.float64)
        done = int(lat.size)
        errors = collections.Counter((r.error or "")[:80] for r in requests if r.status == "failed")
        return dict(requests=len(requests), done=done, retries=sum(r.retries for r in requests),
                    errors=dict(errors),
                    failed=sum(r.status == "failed" for r in requests),
                    rejected=sum(r.status == "rejected" for r in requests),
                    cancelled=sum(r.status == "cancelled" for r in requests),
                    p50_ms=float(np.percentile(lat, 50) * 1e3) if done else None,
                    p99_ms=float(np.percentile(lat, 99) * 1e3) if done else None,
                    mean_ms=float(lat.mean() * 1e3) if done else None,
                    views_per_s=done / wall if wall > 0 else None, wall_s=wall,
                    peak_concurrency=self.peak_concurrency, peak_bytes=self.peak_bytes,
                    budget_bytes=self.budget)


# ---------------------------------------------------------------------------
# CUDA executor
# ---------------------------------------------------------------------------
@dataclass
class _Handle:
    slot: int
    request: ServeRequest
    event: object
    keep: dict


class CudaExecutor:
    """Runs requests through gs_render_batch on one CUDA stream per slot.

    Forward requests copy the image back into pinned host memory; fine-tune
    requests compute a summed L2 loss against a seeded target, run the
    backward pass into fresh gradient buffers and copy the loss back.  The
    resident scene is never modified."""

    def __init__(self, scenes, n_slots: int, opts_fwd=None, opts_bwd=None, device="cuda"):
        import torch

        from . import RasterOpts
        self.torch = torch
        self.scenes = scenes
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self.opts_fwd = opts_fwd or RasterOpts(state_format="fp16")
        self.opts_bwd = opts_bwd or RasterOpts(state_format="fp16")
        # (scene, width, height) -> pair capacity learned from views that overflowed
        self.pair_capacity = {}
        # one workspace allocation per slot, grown when a request needs more: big
        # per-request allocations on many streams would strand cached memory
        self.slot_buffers = [None] * n_slots

    def _opts(self, r):
        import dataclasses
        o = self.opts_bwd if r.backward else self.opts_fwd
        key = (r.scene, int(r.camera.width), int(r.camera.height))
        return dataclasses.replace(o, sh_degree=self.scenes[r.scene].sh_degree,
                                   pair_capacity=self.pair_capacity.get(key, o.pair_capacity))

    def memory(self, r) -> int:
        from . import STATE_BYTES, Workspace
        sc = self.scenes[r.scene]
        o = self._opts(r)
        n = Workspace.required_bytes(sc.n, int(r.camera.width), int(r.camera.height), o)
        px = int(r.camera.width) * int(r.camera.height)
        out = px * (12 + STATE_BYTES[o.state_format] + 4)
        if r.backward:
            out += px * 24 + sc.n * 4 * (3 + 3 + 4 + 1 + 3 * (sc.sh_degree + 1) ** 2)
        return int(n) + out + 1024

    def submit(self, r, slot):
        from . import Request, Workspace, render_batch
        torch = self.torch
        st = self.streams[slot]
        sc = self.scenes[r.scene]
        o = self._opts(r)
        H, W = int(r.camera.height), int(r.camera.width)
        with torch.cuda.stream(st):
            need = Workspace.required_bytes(sc.n, W, H, o) + 256
            buf = self.slot_buffers[slot]
            if buf is None or buf.numel() < need:
                self.slot_buffers[slot] = None
                del buf
                buf = torch.empty(need, dtype=torch.uint8, device=self.device)
                self.slot_buffers[slot] = buf
            ws = Workspace(sc.n, W, H, o, device=self.device, buffer=buf)
            keep = dict(ws=ws)
            target = None
            if r.backward:
                g = torch.Generator(device=self.device)
                g.manual_seed(int(r.target_seed))
                target = torch.rand((H, W, 3), generator=g, device=self.device)
            req = Request(sc, r.camera, o, backward=r.backward,
                          loss_kind="l2" if r.backward else None, target=target)
            render_batch([req], ws, stream=st)
            keep["req"], keep["target"] = req, target
            out = req.outputs
            if r.backward:
                host = torch.empty(1, dtype=torch.float64, pin_memory=True)
                host.copy_(out["loss"], non_blocking=True)
                keep["host_loss"] = host
            else:
                host = torch.empty(out["image"].shape, dtype=torch.float32, pin_memory=True)
                host.copy_(out["image"], non_blocking=True)
                keep["host_image"] = host
            ev = torch.cuda.Event()
            ev.record(st)
        return _Handle(slot, r, ev, keep)

    def poll(self, h) -> bool:
        return h.event.query()

    def finish(self, h) -> dict:
        from . import GsError, check_status, read_counters, _lib
        k = h.keep
        try:
            check_status(k["ws"], stream=self.streams[h.slot])   # device-side errors surface here
        except GsError as e:
            if e.code != _lib.GS_ERR_CAPACITY:
                raise
            want = read_counters(k["ws"], stream=self.streams[h.slot])["pairs_wanted"]
            r = h.request
            key = (r.scene, int(r.camera.width), int(r.camera.height))
            cap = min((1 << 30) - 1, int(want * 1.25) + 4096)
            if want >= (1 << 30) - 1 or cap <= self.pair_capacity.get(key, 0):
                raise
            self.pair_capacity[key] = cap
            raise Retry() from e
        out = k["req"].outputs
        res = dict(image=out["image"])
        if h.request.backward:
            res["loss"] = float(k["host_loss"].item())
            res["grads"] = out["grads"]
        else:
            res["host_image"] = k["host_image"]
        return res


def make_requests(specs, cameras_for):
    """ServeRequest list from dicts of synthetic.serving_requests()."""
    out = []
    for i, s in enumerate(specs):
        out.append(ServeRequest(rid=i, scene=s["scene"], camera=cameras_for(s), backward=s["backward"],
                                arrival=s["arrival"], target_seed=10_000 + i))
    return out
