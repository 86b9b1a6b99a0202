"""The torch.autograd wrapper (GSRender) against the FP64 oracle: analytic
gradients, central finite differences (h = 1e-4) of the oracle's forward, the
activation chain, workspace reuse between forward and backward, and a few
Adam steps."""
import numpy as np
import pytest
import torch

import oracle
import paper_2505_18764_gb300 as gs
from paper_2505_18764_gb300 import autograd as ga
import synthetic as syn
from gpu_helpers import GROUPS, oracle_opts, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    assert torch.cuda.is_available()
    from paper_2505_18764_gb300 import build
    build.build_library()


def _params(scene_np, requires_grad=True):
    return [torch.tensor(a, dtype=torch.float32, device="cuda", requires_grad=requires_grad)
            for a in scene_np.arrays()]


def test_autograd_matches_oracle_and_finite_differences():
    scene_np, cam = syn.gradcheck_subscene()
    opts = gs.RasterOpts(sh_degree=3, t_cull=0.0)
    ws = gs.Workspace(scene_np.n, cam.width, cam.height, opts)
    g = syn.uniform_image(cam.height, cam.width, seed=501, lo=-1.0, hi=1.0)
    params = _params(scene_np)
    img = ga.render(*params, cam, opts, ws)
    loss = (img * torch.from_numpy(g).cuda()).sum()
    loss.backward()
    an = {k: p.grad.cpu().numpy().astype(np.float64) for k, p in zip(GROUPS, params)}
    oo = oracle_opts(opts, cam)
    ref = oracle.backward(scene_np, cam, g.astype(np.float64), oo)
    for k in GROUPS:
        assert rel_l2(an[k], ref[k]) <= 1e-3, k
    # central differences of the FP64 oracle forward on sampled coordinates,
    # skipping any whose +-h perturbation changes a pixel's fragment set
    h = 1e-4
    rng = np.random.default_rng(502)
    base = [a.astype(np.float64) for a in scene_np.arrays()]
    n0 = oracle.render(scene_np, cam, oo)["nfrag"]
    checked = {k: ([], []) for k in GROUPS}
    for gi, k in enumerate(GROUPS):
        flat_n = base[gi].size
        for idx in rng.choice(flat_n, size=min(40, flat_n), replace=False):
            vals, frags = [], []
            for sgn in (+1, -1):
                arr = [b.copy() for b in base]
                arr[gi].reshape(-1)[idx] += sgn * h
                sc = syn.Scene(*arr, scene_np.sh_degree)
                r = oracle.render(sc, cam, oo)
                vals.append(np.sum(r["color"] * g))
                frags.append(r["nfrag"])
            if not (np.array_equal(frags[0], n0) and np.array_equal(frags[1], n0)):
                continue
            checked[k][0].append((vals[0] - vals[1]) / (2 * h))
            checked[k][1].append(an[k].reshape(-1)[idx])
    for k in GROUPS:
        fd, a = np.array(checked[k][0]), np.array(checked[k][1])
        assert len(fd) >= 20, f"{k}: only {len(fd)} clean coordinates"
        assert rel_l2(a, fd) <= 1e-3, f"{k}: rel-L2 {rel_l2(a, fd):.2e} over {len(fd)} coordinates"


def test_activation_chain():
    scene_np, cam = syn.gradcheck_subscene(seed=45)
    opts = gs.RasterOpts(sh_degree=3)
    ws = gs.Workspace(scene_np.n, cam.width, cam.height, opts)
    g = torch.from_numpy(syn.uniform_image(cam.height, cam.width, seed=503, lo=-1, hi=1)).cuda()
    m, s, q, o, sh = _params(scene_np, requires_grad=False)
    log_s = torch.log(s).requires_grad_(True)
    logit = torch.logit(o.double()).float().requires_grad_(True)
    img = ga.render_activated(m, log_s, q, logit, sh, cam, opts, ws)
    (img * g).sum().backward()
    s2, o2 = torch.exp(log_s.detach()), torch.sigmoid(logit.detach())
    img2 = ga.render(m, s2.requires_grad_(True), q, o2.requires_grad_(True), sh, cam, opts, ws)
    (img2 * g).sum().backward()
    torch.testing.assert_close(log_s.grad, s2.grad * s2, rtol=1e-5, atol=1e-7)
    torch.testing.assert_close(logit.grad, o2.grad * o2 * (1 - o2), rtol=1e-5, atol=1e-7)


def test_backward_after_workspace_reuse():
    scene_np, cams = syn.precision_sweep_views(2)
    opts = gs.RasterOpts()
    ws = gs.Workspace(scene_np.n, 128, 128, opts)
    g = torch.from_numpy(syn.uniform_image(128, 128, seed=504, lo=-1, hi=1)).cuda()
    pa = _params(scene_np)
    img_a = ga.render(*pa, cams[0], opts, ws)
    pb = _params(scene_np)
    img_b = ga.render(*pb, cams[1], opts, ws)      # overwrites the workspace
    (img_a * g).sum().backward()                    # must redo view A's preparation
    (img_b * g).sum().backward()
    pc = _params(scene_np)
    img_c = ga.render(*pc, cams[0], opts, ws)
    (img_c * g).sum().backward()
    # the per-splat sums are atomic adds in an order that varies run to run:
    # equal up to FP32 reassociation
    for x, y in zip(pa, pc):
        err = (x.grad - y.grad).norm() / y.grad.norm().clamp_min(1e-30)
        assert err < 1e-5, float(err)
    assert torch.equal(img_a, img_c)


def test_adam_steps_reduce_l2_loss():
    scene_np = syn.cube_scene(2000, seed=4, sh_degree=3)
    cams = [syn.orbit_camera(2 * np.pi * k / 4, 4.0, 60.0, 96, 72) for k in range(4)]
    targets = [torch.from_numpy(syn.uniform_image(72, 96, seed=600 + k)).cuda() for k in range(4)]
    model = ga.Renderer(scene_np, 96, 72, gs.RasterOpts(sh_degree=3, state_format="fp16"))
    opt = torch.optim.Adam(model.parameters(), lr=1e-3)
    losses = []
    for it in range(12):
        opt.zero_grad()
        loss = sum(((model(c) - t) ** 2).sum() for c, t in zip(cams, targets))
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert np.isfinite(losses).all() and losses[-1] < losses[0]
