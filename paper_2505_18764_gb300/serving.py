"""Continuous-batching render server.

Scenes stay resident on the device.  Requests (a novel-view render, or a
forward + backward fine-tune step that returns the loss and the per-splat
gradients without changing the resident scene) arrive over time.  The
scheduler admits the oldest waiting request as soon as a slot is free and its
device memory (workspace + outputs, computed exactly from gs_workspace_size)
fits under the HBM budget; admitted requests run on their slot's own CUDA
stream, so work that arrives while others are on the GPU overlaps with them.
Latency = completion - arrival; the server reports p50 / p99 latency (and the
admit-to-done service time) and views per second.

An executor may offer several plans for a request, fastest first, each with
its device memory: the CUDA executor offers the single-pass render and the
memory-efficiency mode (the view binned and rasterized in chunks of the depth
order under a small pair capacity, Sec. 4.5), which trades time for memory.
The scheduler runs the first plan that fits the budget left; a request whose
smallest plan exceeds the whole budget is rejected.

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
    plan: object = None          # the executor's plan the request ran with
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

    def _plans(self, r):
        """[(bytes, plan)] in the executor's order of preference (fastest first)."""
        if hasattr(self.ex, "plans"):
            return list(self.ex.plans(r))
        return [(self.ex.memory(r), None)]

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
                plans = self._plans(r)
                smallest = min(b for b, _ in plans)
                if smallest > self.budget:
                    waiting.popleft()
                    r.status, r.error = "rejected", f"needs {smallest} B, budget {self.budget} B"
                    progressed = True
                    continue
                fit = [(b, p) for b, p in plans if self.in_flight_bytes + b <= self.budget]
                if not fit:
                    break  # wait for memory to free up
                need, plan = fit[0]
                waiting.popleft()
                slot = free_slots.pop()
                r.t_admit = time.perf_counter() - t0
                r.status = "running"
                r.plan = plan
                try:
                    h = self.ex.submit(r, slot) if plan is None else self.ex.submit(r, slot, plan)
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
        svc = np.array([r.t_done - r.t_admit for r in requests if r.status == "done"],
                       dtype=np.float64)
        done = int(lat.size)
        half = len(requests) // 2
        first = [r.latency for r in requests[:half] if r.status == "done"]
        second = [r.latency for r in requests[half:] if r.status == "done"]
        plans = collections.Counter(str(r.plan) for r in requests if r.status == "done")
        errors = collections.Counter((r.error or "")[:80] for r in requests if r.status == "failed")
        return dict(requests=len(requests), done=done, retries=sum(r.retries for r in requests),
                    errors=dict(errors),
                    failed=sum(r.status == "failed" for r in requests),
                    rejected=sum(r.status == "rejected" for r in requests),
                    cancelled=sum(r.status == "cancelled" for r in requests),
                    p50_ms=float(np.percentile(lat, 50) * 1e3) if done else None,
                    p99_ms=float(np.percentile(lat, 99) * 1e3) if done else None,
                    mean_ms=float(lat.mean() * 1e3) if done else None,
                    service_p50_ms=float(np.percentile(svc, 50) * 1e3) if done else None,
                    service_p99_ms=float(np.percentile(svc, 99) * 1e3) if done else None,
                    p99_first_half_ms=float(np.percentile(first, 99) * 1e3) if first else None,
                    p99_second_half_ms=float(np.percentile(second, 99) * 1e3) if second else None,
                    plans=dict(plans),
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
    resident scene is never modified.

    Plans: "single" (one pass; the pair capacity learned from views that
    overflowed) and "chunked" (the memory-efficiency mode with a pair capacity
    of `chunk_pairs`, at least twice the view's block count), offered when it
    needs less memory.  With reuse_outputs, each slot keeps its output and
    pinned host buffers from request to request (a result is valid until the
    slot's next request: for a server that delivers results before reusing a
    slot); otherwise every request gets fresh ones."""

    def __init__(self, scenes, n_slots: int, opts_fwd=None, opts_bwd=None, device="cuda",
                 chunk_pairs: int = 1 << 20, reuse_outputs: bool = False):
        import torch

        from . import RasterOpts
        self.torch = torch
        self.scenes = scenes
        self.device = torch.device(device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(n_slots)]
        self.opts_fwd = opts_fwd or RasterOpts(state_format="fp16")
        self.opts_bwd = opts_bwd or RasterOpts(state_format="fp16")
        self.chunk_pairs = int(chunk_pairs)
        self.reuse = bool(reuse_outputs)
        # (scene, width, height) -> pair capacity learned from views that overflowed
        self.pair_capacity = {}
        # one workspace allocation per slot, grown when a request needs more: big
        # per-request allocations on many streams would strand cached memory
        self.slot_buffers = [None] * n_slots
        self.slot_outputs = [dict() for _ in range(n_slots)]
        self.gpu_ms = []   # device time of each finished request (events on its stream)

    def _opts(self, r, plan="single"):
        import dataclasses
        o = self.opts_bwd if r.backward else self.opts_fwd
        o = dataclasses.replace(o, sh_degree=self.scenes[r.scene].sh_degree)
        if plan == "chunked":
            blocks = ((int(r.camera.width) + 15) // 16) * ((int(r.camera.height) + 15) // 16)
            return dataclasses.replace(o, chunked=True,
                                       pair_capacity=max(self.chunk_pairs, 2 * blocks + 4096))
        key = (r.scene, int(r.camera.width), int(r.camera.height))
        return dataclasses.replace(o, pair_capacity=self.pair_capacity.get(key, o.pair_capacity))

    def _bytes(self, r, o) -> int:
        from . import STATE_BYTES, Workspace
        sc = self.scenes[r.scene]
        n = Workspace.required_bytes(sc.n, int(r.camera.width), int(r.camera.height), o)
        px = int(r.camera.width) * int(r.camera.height)
        out = px * (12 + STATE_BYTES[o.state_format] + 4)
        if r.backward:
            out += px * 24 + sc.n * 4 * (3 + 3 + 4 + 1 + 3 * (sc.sh_degree + 1) ** 2)
        return int(n) + out + 1024

    def memory(self, r) -> int:
        """Device memory of the single-pass plan."""
        return self._bytes(r, self._opts(r))

    def plans(self, r):
        single = self.memory(r)
        chunked = self._bytes(r, self._opts(r, "chunked"))
        return [(single, "single")] + ([(chunked, "chunked")] if chunked < single else [])

    def _slot_tensor(self, slot, name, shape, dtype, pinned=False):
        """A view of the slot's buffer `name` (grown as needed) of `shape`."""
        torch = self.torch
        numel = 1
        for d in shape:
            numel *= int(d)
        buf = self.slot_outputs[slot].get(name)
        if buf is None or buf.numel() < numel or buf.dtype != dtype:
            buf = (torch.empty(numel, dtype=dtype, pin_memory=True) if pinned else
                   torch.empty(numel, dtype=dtype, device=self.device))
            self.slot_outputs[slot][name] = buf
        return buf[:numel].view(*shape)

    def submit(self, r, slot, plan="single"):
        from . import STATE_BYTES, Request, Workspace, render_batch
        torch = self.torch
        st = self.streams[slot]
        sc = self.scenes[r.scene]
        o = self._opts(r, plan)
        H, W = int(r.camera.height), int(r.camera.width)
        with torch.cuda.stream(st):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev0.record(st)
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
            if self.reuse:
                out = req.outputs
                out["image"] = self._slot_tensor(slot, "image", (H, W, 3), torch.float32)
                out["state"] = self._slot_tensor(slot, "state", (H, W, STATE_BYTES[o.state_format]),
                                                 torch.uint8)
                out["last"] = self._slot_tensor(slot, "last", (H, W), torch.int32)
                if r.backward:
                    out["dL_dimage"] = self._slot_tensor(slot, "dl", (H, W, 3), torch.float32)
                    out["loss"] = self._slot_tensor(slot, "loss", (1,), torch.float64)
            render_batch([req], ws, stream=st)
            keep["req"], keep["target"] = req, target
            out = req.outputs
            if r.backward:
                host = (self._slot_tensor(slot, "host_loss", (1,), torch.float64, pinned=True)
                        if self.reuse else torch.empty(1, dtype=torch.float64, pin_memory=True))
                host.copy_(out["loss"], non_blocking=True)
                keep["host_loss"] = host
            else:
                host = (self._slot_tensor(slot, "host_image", (H, W, 3), torch.float32, pinned=True)
                        if self.reuse else
                        torch.empty(out["image"].shape, dtype=torch.float32, pin_memory=True))
                host.copy_(out["image"], non_blocking=True)
                keep["host_image"] = host
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(st)
            keep["ev0"] = ev0
        return _Handle(slot, r, ev, keep)

    def poll(self, h) -> bool:
        return h.event.query()

    def finish(self, h) -> dict:
        from . import GsError, check_status, read_counters, _lib
        k = h.keep
        self.gpu_ms.append(k["ev0"].elapsed_time(h.event))
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
