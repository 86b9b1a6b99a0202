"""The render server on the GPU: each request's result is the same alone and
in an overlapping mix (images bit-identical, losses and gradients within FP32
reassociation of the atomic gradient sums), and admission keeps the in-flight
device memory under the budget."""
import numpy as np
import pytest
import torch

import paper_2505_18764_gb300 as gs
from paper_2505_18764_gb300.serving import CudaExecutor, Server, ServeRequest
import synthetic as syn

pytestmark = pytest.mark.gpu


def _setup():
    from paper_2505_18764_gb300 import build
    build.build_library()
    scenes = [gs.SceneTensors.from_numpy(syn.cube_scene(n, seed=70 + n % 7, sh_degree=3))
              for n in (20_000, 60_000)]
    sizes = [(96, 64), (160, 120), (200, 150)]
    rng = np.random.default_rng(71)
    reqs = []
    for i in range(24):
        w, h = sizes[i % 3]
        cam = syn.orbit_camera(float(rng.uniform(0, 2 * np.pi)), 4.0, 60.0, w, h)
        reqs.append(ServeRequest(rid=i, scene=i % 2, camera=cam, backward=(i % 4 == 1),
                                 arrival=0.0, target_seed=900 + i))
    return scenes, reqs


def _clone(reqs):
    return [ServeRequest(rid=r.rid, scene=r.scene, camera=r.camera, backward=r.backward,
                         arrival=r.arrival, target_seed=r.target_seed) for r in reqs]


def test_results_identical_alone_and_in_the_mix():
    scenes, reqs = _setup()
    mixed = _clone(reqs)
    srv = Server(CudaExecutor(scenes, 4), hbm_budget_bytes=8 << 30, max_slots=4)
    stats = srv.run(mixed, realtime=False)
    assert stats["done"] == len(reqs) and srv.peak_concurrency > 1
    torch.cuda.synchronize()
    for r in reqs:                        # one at a time, one slot
        alone = _clone([r])
        Server(CudaExecutor(scenes, 1), hbm_budget_bytes=8 << 30, max_slots=1).run(alone, realtime=False)
        a, m = alone[0].result, mixed[r.rid].result
        assert alone[0].status == "done"
        assert torch.equal(a["image"], m["image"])
        if r.backward:
            assert abs(a["loss"] - m["loss"]) <= 1e-9 * abs(a["loss"])
            for k in ("means", "scales", "quats", "opacities", "sh"):
                x, y = a["grads"][k].double(), m["grads"][k].double()
                assert (torch.linalg.norm(x - y) / torch.linalg.norm(x)).item() < 1e-5, k
        else:
            assert torch.equal(a["host_image"], m["host_image"])


def test_budget_admission_on_gpu():
    scenes, reqs = _setup()
    ex = CudaExecutor(scenes, 4)
    mem = sorted(ex.memory(r) for r in reqs)
    budget = mem[-1] + mem[0] // 2          # the largest request never overlaps another
    srv = Server(ex, hbm_budget_bytes=budget, max_slots=4)
    stats = srv.run(_clone(reqs), realtime=False)
    assert stats["done"] == len(reqs)
    assert srv.peak_bytes <= budget and srv.peak_concurrency < 4


def test_chunked_plan_under_a_tight_budget_matches_the_request_alone():
    """A budget below every request's single-pass memory makes the server run
    them in the memory-efficiency mode; with FP32 state the chunked render is
    the single-pass render bit for bit, and the fine-tune gradients agree to
    FP32 reassociation."""
    scenes, reqs = _setup()
    opts = gs.RasterOpts(state_format="fp32")
    ex = CudaExecutor(scenes, 2, opts_fwd=opts, opts_bwd=opts, chunk_pairs=1 << 12)
    plans = [ex.plans(r) for r in reqs]
    assert all(len(p) == 2 for p in plans)
    budget = max(p[1][0] for p in plans) + 1024       # fits every chunked plan, no single one
    assert budget < min(p[0][0] for p in plans)
    chunked = _clone(reqs)
    stats = Server(ex, hbm_budget_bytes=budget, max_slots=2).run(chunked, realtime=False)
    assert stats["done"] == len(reqs) and stats["plans"] == {"chunked": len(reqs)}
    for r in reqs:
        alone = _clone([r])
        Server(CudaExecutor(scenes, 1, opts_fwd=opts, opts_bwd=opts), hbm_budget_bytes=8 << 30,
               max_slots=1).run(alone, realtime=False)
        a, c = alone[0].result, chunked[r.rid].result
        assert alone[0].plan == "single"
        assert torch.equal(a["image"], c["image"])
        if r.backward:
            assert abs(a["loss"] - c["loss"]) <= 1e-9 * abs(a["loss"])
            for k in ("means", "scales", "quats", "opacities", "sh"):
                x, y = a["grads"][k].double(), c["grads"][k].double()
                assert (torch.linalg.norm(x - y) / torch.linalg.norm(x)).item() < 1e-5, k
