"""Pins for the FP64 oracle, checked against things other than itself:
library special functions, closed forms, invariants, brute force and finite
differences.  CPU only."""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn

Y00 = 0.5 / math.sqrt(math.pi)  # textbook value of Y_0^0


# ---------------------------------------------------------------------------
# Spherical harmonics (colour model of Sec. 2.1.1)
# ---------------------------------------------------------------------------

def _real_sh_scipy(l, m, dirs):
    """Real SH from scipy's complex Y_l^m (Condon-Shortley phase included)."""
    from scipy.special import sph_harm_y
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    theta = np.arccos(np.clip(z, -1.0, 1.0))
    phi = np.mod(np.arctan2(y, x), 2.0 * np.pi)
    Yc = sph_harm_y(l, abs(m), theta, phi)
    if m == 0:
        return Yc.real
    if m > 0:
        return math.sqrt(2.0) * Yc.real
    return math.sqrt(2.0) * Yc.imag


def _rand_dirs(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.standard_normal((n, 3))
    return d / np.linalg.norm(d, axis=1, keepdims=True)


def test_sh_matches_scipy_real_basis():
    dirs = _rand_dirs(200, 0)
    Y = oracle.sh_basis(3, dirs)
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_sh_scipy(l, m, dirs)
            np.testing.assert_allclose(Y[:, l * l + l + m], ref, rtol=0, atol=1e-12)


def test_sh_orthonormal_by_quadrature():
    zs, wz = np.polynomial.legendre.leggauss(16)
    nphi = 16
    phis = 2.0 * np.pi * np.arange(nphi) / nphi
    Z, P = np.meshgrid(zs, phis, indexing="ij")
    rho = np.sqrt(1.0 - Z ** 2)
    dirs = np.stack([rho * np.cos(P), rho * np.sin(P), Z], axis=-1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2.0 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle.sh_basis(3, dirs)
    gram = (Y * w[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_textbook_values():
    # Y_0^0, Y_1^{-1,0,1} at the axes (Condon-Shortley: Y_1^1 = -sqrt(3/4pi) x).
    c1 = math.sqrt(3.0 / (4.0 * math.pi))
    Y = oracle.sh_basis(1, np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]]))
    np.testing.assert_allclose(Y[:, 0], Y00, atol=1e-15)
    np.testing.assert_allclose(Y[0, 1:], [0.0, 0.0, -c1], atol=1e-15)
    np.testing.assert_allclose(Y[1, 1:], [-c1, 0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(Y[2, 1:], [0.0, c1, 0.0], atol=1e-15)


def test_sh_addition_theorem():
    # sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) P_l(a . b)
    a, b = _rand_dirs(50, 1), _rand_dirs(50, 2)
    Ya, Yb = oracle.sh_basis(3, a), oracle.sh_basis(3, b)
    cosg = np.sum(a * b, axis=1)
    for l in range(4):
        s = np.sum(Ya[:, l * l:(l + 1) ** 2] * Yb[:, l * l:(l + 1) ** 2], axis=1)
        Pl = np.polynomial.legendre.legval(cosg, [0] * l + [1])
        np.testing.assert_allclose(s, (2 * l + 1) / (4 * math.pi) * Pl, atol=1e-12)


def test_sh_tangential_gradient_matches_fd():
    dirs = _rand_dirs(40, 3)
    Y, dY = oracle.sh_basis(3, dirs, grad=True)
    h = 1e-6
    rng = np.random.default_rng(4)
    for _ in range(3):
        v = rng.standard_normal((40, 3))
        v -= dirs * np.sum(v * dirs, axis=1, keepdims=True)  # tangent direction
        p = dirs + h * v
        m = dirs - h * v
        p /= np.linalg.norm(p, axis=1, keepdims=True)
        m /= np.linalg.norm(m, axis=1, keepdims=True)
        fd = (oracle.sh_basis(3, p) - oracle.sh_basis(3, m)) / (2 * h)
        an = np.einsum("nkj,nj->nk", dY, v)
        np.testing.assert_allclose(an, fd, atol=2e-7)


# ---------------------------------------------------------------------------
# Projection (Sec. 2.1.2)
# ---------------------------------------------------------------------------

def _one_splat(mu, scale, quat, opac, rgb, deg=0):
    K = (deg + 1) ** 2
    sh = np.zeros((1, K, 3), np.float32)
    sh[0, 0, :] = (np.asarray(rgb) - 0.5) / Y00
    return syn.Scene(np.array([mu], np.float32), np.array([scale], np.float32),
                     np.array([quat], np.float32), np.array([opac], np.float32), sh, deg)


def _quat_rotate(q, v):
    """Rotate v by unit quaternion q = (w, x, y, z) with Hamilton products q v q*."""
    def mul(a, b):
        w1, x1, y1, z1 = a
        w2, x2, y2, z2 = b
        return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                         w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                         w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                         w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])
    qc = q * np.array([1, -1, -1, -1])
    return mul(mul(q, np.concatenate([[0.0], v])), qc)[1:]


def test_projection_sigma2d_against_independent_route():
    cam = syn.look_at((0.3, -0.2, -4.0), (0.0, 0.1, 0.0), 50.0, 96, 64)
    rng = np.random.default_rng(5)
    for trial in range(5):
        mu = rng.uniform(-0.8, 0.8, 3)
        s = np.exp(rng.normal(-2.0, 0.4, 3))
        q = rng.standard_normal(4)
        sc = _one_splat(mu, s, q, 0.8, (0.2, 0.5, 0.7))
        out = oracle.project(sc, cam)[0]
        mu64, s64, q64 = (sc.means[0].astype(np.float64), sc.scales[0].astype(np.float64),
                          sc.quats[0].astype(np.float64))
        qn = q64 / np.linalg.norm(q64)
        R = np.stack([_quat_rotate(qn, e) for e in np.eye(3)], axis=1)  # columns = R e_j
        S3 = R @ np.diag(s64 ** 2) @ R.T
        V = cam.viewmat.astype(np.float64)
        W, w = V[:, :3], V[:, 3]
        fx, fy, cx, cy = cam.fx, cam.fy, cam.cx, cam.cy

        def proj(t):
            return np.array([fx * t[0] / t[2] + cx, fy * t[1] / t[2] + cy])

        t = W @ mu64 + w
        h = 1e-6
        J = np.stack([(proj(t + h * e) - proj(t - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        S2 = J @ W @ S3 @ W.T @ J.T + 0.3 * np.eye(2)
        assert out[0] == 1.0
        np.testing.assert_allclose(out[1:3], proj(t), rtol=1e-13)
        np.testing.assert_allclose(out[[3, 4, 5]], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-7, atol=1e-9)
        Q = np.linalg.inv(S2)
        np.testing.assert_allclose(out[[6, 7, 8]], [Q[0, 0], Q[0, 1], Q[1, 1]], rtol=1e-7, atol=1e-9)
        np.testing.assert_allclose(out[12], t[2], rtol=1e-14)


def test_near_plane_and_zero_quaternion_invalid():
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 60.0, 32, 32)
    # world z = -3.85 -> camera depth 0.15 < 0.2
    sc = _one_splat((0.0, 0.0, -3.85), (0.1, 0.1, 0.1), (1, 0, 0, 0), 0.9, (1, 1, 1))
    assert oracle.project(sc, cam)[0, 0] == 0.0
    sc = _one_splat((0.0, 0.0, 0.0), (0.1, 0.1, 0.1), (0, 0, 0, 0), 0.9, (1, 1, 1))
    assert oracle.project(sc, cam)[0, 0] == 0.0
    img = oracle.render(sc, cam)["color"]
    assert np.all(img == 0.0)


# ---------------------------------------------------------------------------
# Forward compositing (Eq. 2, alpha floor, alpha clamp, T-culling)
# ---------------------------------------------------------------------------

def test_single_isotropic_splat_closed_form():
    W = H = 48
    fov = 50.0
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), fov, W, H)
    f = np.float64(np.float32(H / (2 * math.tan(math.radians(fov) / 2))))
    s = np.float64(np.float32(0.12))
    o = np.float64(np.float32(0.8))
    rgb = np.array([0.9, 0.4, 0.1])
    sc = _one_splat((0.0, 0.0, 0.0), (s, s, s), (1.0, 0.0, 0.0, 0.0), o, rgb)
    rgb_in = sc.sh[0, 0].astype(np.float64) * Y00 + 0.5
    res = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0))
    sigma2 = (f * s / 4.0) ** 2 + 0.3
    ys, xs = np.mgrid[0:H, 0:W] + 0.5
    d2 = (xs - W / 2) ** 2 + (ys - H / 2) ** 2
    alpha = np.minimum(0.99, o * np.exp(-d2 / (2 * sigma2)))
    alpha = np.where(alpha >= 1.0 / 255.0, alpha, 0.0)
    np.testing.assert_allclose(res["color"], alpha[..., None] * rgb_in[None, None, :], atol=1e-12)
    np.testing.assert_allclose(res["T"], 1.0 - alpha, atol=1e-12)
    np.testing.assert_array_equal(res["nfrag"], (alpha > 0).astype(np.int32))
    np.testing.assert_array_equal(res["last"], np.where(alpha > 0, 0, -1))


def test_alpha_clamp_and_floor():
    W = H = 16
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 50.0, W, H)
    # huge splat with o = 1: alpha = min(0.99, ~1) = 0.99 at the centre
    sc = _one_splat((0.0, 0.0, 0.0), (2.0, 2.0, 2.0), (1, 0, 0, 0), 1.0, (1.0, 1.0, 1.0))
    res = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0))
    assert abs(res["T"][H // 2, W // 2] - 0.01) < 1e-12
    rgb_in = sc.sh[0, 0].astype(np.float64) * Y00 + 0.5
    assert np.all(res["color"] <= 0.99 * rgb_in[None, None, :] * (1 + 1e-15))
    # opacity just under 1/255: no fragment anywhere
    sc = _one_splat((0.0, 0.0, 0.0), (2.0, 2.0, 2.0), (1, 0, 0, 0), 0.999 / 255.0, (1, 1, 1))
    res = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0))
    assert res["nfrag"].sum() == 0 and np.all(res["color"] == 0.0)


def test_two_splat_occlusion_order():
    W = H = 32
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 50.0, W, H)
    front = dict(mu=(0.0, 0.0, -1.0), s=0.3, o=0.7, rgb=(1.0, 0.0, 0.0))
    back = dict(mu=(0.0, 0.0, 1.0), s=0.3, o=0.9, rgb=(0.0, 0.0, 1.0))
    for order in ((front, back), (back, front)):
        sh = np.zeros((2, 1, 3), np.float32)
        for i, sp in enumerate(order):
            sh[i, 0] = (np.array(sp["rgb"]) - 0.5) / Y00
        sc = syn.Scene(np.array([sp["mu"] for sp in order], np.float32),
                       np.array([[sp["s"]] * 3 for sp in order], np.float32),
                       np.array([[1, 0, 0, 0]] * 2, np.float32),
                       np.array([sp["o"] for sp in order], np.float32), sh, 0)
        res = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0))
        P = oracle.project(sc, cam)
        c = res["color"][H // 2, W // 2]
        ux = uy = W // 2 + 0.5
        a = []
        for i in range(2):
            d = np.array([ux - P[i, 1], uy - P[i, 2]])
            Q = np.array([[P[i, 6], P[i, 7]], [P[i, 7], P[i, 8]]])
            a.append(min(0.99, np.float64(order[i]["o"] if False else sc.opacities[i]) *
                         math.exp(-0.5 * d @ Q @ d)))
        fi = 0 if order[0] is front else 1
        bi = 1 - fi
        rgb = P[:, 9:12]
        expect = a[fi] * rgb[fi] + (1 - a[fi]) * a[bi] * rgb[bi]
        np.testing.assert_allclose(c, expect, atol=1e-13)


def test_opaque_front_and_t_culling():
    W = H = 8
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 50.0, W, H)
    n = 4
    sh = np.zeros((n, 1, 3), np.float32)
    sh[:, 0, :] = (1.0 - 0.5) / Y00
    sc = syn.Scene(np.array([[0, 0, z] for z in (-1.5, -0.5, 0.5, 1.5)], np.float32),
                   np.full((n, 3), 10.0, np.float32), np.array([[1, 0, 0, 0]] * n, np.float32),
                   np.ones(n, np.float32), sh, 0)
    r0 = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0))
    assert r0["nfrag"][H // 2, W // 2] == 4
    assert r0["T"][H // 2, W // 2] <= 0.01 ** 4 * (1 + 1e-9)
    # T_1 = 1, T_2 = 0.01, T_3 = 1e-4, T_4 = 1e-6 < 5e-5: the fourth fragment is skipped
    r1 = oracle.render(sc, cam, oracle.opts_array(t_cull=5e-5))
    assert r1["nfrag"][H // 2, W // 2] == 3
    assert abs(r1["T"][H // 2, W // 2] - 1e-6) < 1e-12
    assert r1["last"][H // 2, W // 2] == 2


def test_invariants_on_tiny_scene():
    scene, cam, _ = syn.tiny_scene_1k()
    r = oracle.render(scene, cam)
    T = r["T"]
    assert np.all(T >= 0.0) and np.all(T <= 1.0)
    assert np.all(r["color"] >= 0.0)
    # fragments exist and the scene covers a good share of the image
    assert r["nfrag"].sum() > 10000
    assert (r["nfrag"] > 0).mean() > 0.3


def test_brute_force_coverage_and_color():
    """Per-pixel fragment sets against an all-pixels x all-splats numpy evaluation."""
    scene = syn.cube_scene(128, seed=7, sh_degree=1, log_scale_mean=-2.5)
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 50.0, 40, 36)
    r = oracle.render(scene, cam, oracle.opts_array(t_cull=0.0))
    P = oracle.project(scene, cam)
    valid = P[:, 0] == 1.0
    order = np.argsort(P[:, 12], kind="stable")
    order = order[valid[order]]
    ys, xs = np.mgrid[0:cam.height, 0:cam.width] + 0.5
    ux, uy = xs.reshape(-1, 1), ys.reshape(-1, 1)
    dx, dy = ux - P[order, 1][None], uy - P[order, 2][None]
    power = -0.5 * (P[order, 6] * dx * dx + 2 * P[order, 7] * dx * dy + P[order, 8] * dy * dy)
    alpha = np.minimum(0.99, scene.opacities[order].astype(np.float64)[None] * np.exp(power))
    frag = alpha >= 1.0 / 255.0
    a = np.where(frag, alpha, 0.0)
    Tb = np.cumprod(np.concatenate([np.ones((a.shape[0], 1)), 1.0 - a[:, :-1]], axis=1), axis=1)
    C = np.einsum("pk,kc->pc", Tb * a, P[order, 9:12])
    np.testing.assert_array_equal(r["nfrag"].reshape(-1), frag.sum(axis=1))
    np.testing.assert_allclose(r["color"].reshape(-1, 3), C, atol=1e-12)


def test_pixel_subset_matches_full_render():
    scene, cam, _ = syn.tiny_scene_1k()
    full = oracle.render(scene, cam)
    rng = np.random.default_rng(8)
    pix = rng.choice(cam.width * cam.height, size=300, replace=False)
    sub = oracle.render(scene, cam, pixels=pix)
    np.testing.assert_array_equal(sub["color"], full["color"].reshape(-1, 3)[pix])
    np.testing.assert_array_equal(sub["nfrag"], full["nfrag"].reshape(-1)[pix])


def test_stable_sort_against_numpy():
    rng = np.random.default_rng(9)
    keys = rng.integers(0, 50, size=5000).astype(np.uint32)
    np.testing.assert_array_equal(oracle.stable_sort_u32(keys), np.argsort(keys, kind="stable"))


@pytest.mark.parametrize("fmt", ["fp16", "unorm16", "unorm8"])
def test_store_only_rounding_matches_numpy(fmt):
    scene, cam, _ = syn.tiny_scene_1k()
    exact = oracle.render(scene, cam, oracle.opts_array(clamp01=True))
    q = oracle.render(scene, cam, oracle.opts_array(clamp01=True, quant=oracle.QUANT[fmt]))
    c = exact["color"]
    if fmt == "fp16":
        ref = c.astype(np.float16).astype(np.float64)
    else:
        s = 65535.0 if fmt == "unorm16" else 255.0
        ref = np.round(np.clip(c, 0, 1) * s) / s
    np.testing.assert_array_equal(q["color"], ref)


# ---------------------------------------------------------------------------
# Backward: Eq. 3 / Eq. 4 and the chain rule, against central differences
# ---------------------------------------------------------------------------

def _fd_scene(seed, n=6, deg=3, size=24, opaque=False):
    sc = syn.cube_scene(n, seed=seed, sh_degree=deg, log_scale_mean=-1.6, log_scale_std=0.3,
                        extent=0.6, hi_sigma=0.15)
    if opaque:
        sc.opacities[0] = 1.0
        sc.scales[0] = np.array([0.5, 0.4, 0.45], np.float32)
    cam = syn.look_at((0.2, -0.1, -4.0), (0.0, 0.0, 0.0), 40.0, size, size)
    return sc, cam


def _loss(scene, cam, g, opts):
    return float(np.sum(oracle.render(scene, cam, opts)["color"] * g))


def _clean(scene, cam, opts_bands):
    r = oracle.render(scene, cam, opts_bands)
    return not np.any(r["ambig"] & (1 | 4 | 16))


@pytest.mark.parametrize("clamp01,opaque", [(False, False), (True, False), (False, True)])
def test_backward_matches_central_differences(clamp01, opaque):
    bands = dict(band_cut=1e-3, band_clamp=1e-3, band_t=1e-2)
    seed = 100
    while True:
        sc, cam = _fd_scene(seed, opaque=opaque)
        if _clean(sc, cam, oracle.opts_array(t_cull=0.0, clamp01=clamp01, **bands)):
            break
        seed += 1
        assert seed < 400, "no clean fixture found"
    opts = oracle.opts_array(t_cull=0.0, clamp01=clamp01)
    rng = np.random.default_rng(seed)
    g = rng.uniform(-1, 1, size=(cam.height, cam.width, 3))
    an = oracle.backward(sc, cam, g, opts)
    # the scene must exercise the clamp branches this case is about
    if opaque:
        r = oracle.render(sc, cam, opts)
        assert np.min(r["T"]) < 0.02
    h = 1e-6
    # FD in float64 on a float64 copy of the parameters
    base = [a.astype(np.float64) for a in sc.arrays()]
    names = ["means", "scales", "quats", "opacities", "sh"]
    for gi, name in enumerate(names):
        fd = np.zeros_like(base[gi])
        flat = fd.reshape(-1)
        for k in range(flat.size):
            arrs_p = [b.copy() for b in base]
            arrs_m = [b.copy() for b in base]
            arrs_p[gi].reshape(-1)[k] += h
            arrs_m[gi].reshape(-1)[k] -= h
            sp_ = syn.Scene(*arrs_p, sc.sh_degree)
            sm_ = syn.Scene(*arrs_m, sc.sh_degree)
            flat[k] = (_loss(sp_, cam, g, opts) - _loss(sm_, cam, g, opts)) / (2 * h)
        a = an[name]
        err = np.linalg.norm(a - fd) / max(np.linalg.norm(fd), 1e-12)
        assert err < 1e-6, f"{name}: rel-L2 {err:.3e}"
        assert np.linalg.norm(fd) > 1e-6, f"{name}: zero gradient, fixture too weak"


def test_backward_with_t_culling_matches_differences():
    """Four stacked opaque splats and t_cull = 5e-5: the culled fourth fragment
    contributes nothing, and the analytic gradient is that of the culled image."""
    W = H = 12
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 50.0, W, H)
    n = 4
    rng = np.random.default_rng(11)
    sh = rng.normal(0, 0.3, size=(n, 1, 3)).astype(np.float32)
    sc = syn.Scene(np.array([[0.01, -0.02, z] for z in (-1.5, -0.5, 0.5, 1.5)], np.float32),
                   np.array([[0.9, 0.8, 0.85]] * n, np.float32),
                   np.array([[1, 0.05, 0.02, 0]] * n, np.float32),
                   np.array([0.9999] * n, np.float32), sh, 0)
    opts = oracle.opts_array(t_cull=5e-5, band_t=1e-3)
    r = oracle.render(sc, cam, opts)
    r0 = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0))
    culled = r["nfrag"] < r0["nfrag"]
    assert culled.sum() >= 4 and (~culled & (r0["nfrag"] == 4)).sum() >= 4
    assert not np.any(r["ambig"] & 4)
    g = rng.uniform(-1, 1, size=(H, W, 3))
    an = oracle.backward(sc, cam, g, opts)
    an0 = oracle.backward(sc, cam, g, oracle.opts_array(t_cull=0.0))
    assert np.linalg.norm(an["sh"][3] - an0["sh"][3]) > 1e-6  # culling changed the gradient
    base = [a.astype(np.float64) for a in sc.arrays()]
    h = 1e-6
    for gi, name in enumerate(["means", "scales", "opacities", "sh"]):
        gi_ = [0, 1, 3, 4][gi]
        fd = np.zeros_like(base[gi_])
        for k in range(fd.size):
            p = [b.copy() for b in base]
            m = [b.copy() for b in base]
            p[gi_].reshape(-1)[k] += h
            m[gi_].reshape(-1)[k] -= h
            fd.reshape(-1)[k] = (_loss(syn.Scene(*p, 0), cam, g, opts) -
                                 _loss(syn.Scene(*m, 0), cam, g, opts)) / (2 * h)
        err = np.linalg.norm(an[name] - fd) / max(np.linalg.norm(fd), 1e-12)
        assert err < 1e-5, f"{name}: {err:.2e}"
        if name == "sh":
            # the culled fragments' share (~5e-6) is resolved: FD sides with the culled image
            assert np.max(np.abs(an["sh"][3] - fd[3])) < 1e-8
            assert np.max(np.abs(an0["sh"][3] - fd[3])) > 1e-6


def test_eq4_equals_eq7_recurrence_on_fragment_lists():
    """The explicit suffix sum of Eq. 4 equals the front-to-back form of Eq. 7
    with C'_1 = C and C'_{i+1} = C'_i - T_i alpha_i c_i (Eq. 5, Eq. 6)."""
    rng = np.random.default_rng(12)
    for _ in range(20):
        n = rng.integers(1, 30)
        alpha = rng.uniform(1 / 255, 0.99, n)
        c = rng.uniform(0, 1, (n, 3))
        g = rng.uniform(-1, 1, 3)
        T = np.concatenate([[1.0], np.cumprod(1 - alpha)[:-1]])
        w = (T * alpha)[:, None] * c
        S = np.concatenate([np.cumsum(w[::-1], axis=0)[::-1][1:], np.zeros((1, 3))])
        eq4 = np.sum(g * (c * T[:, None] - S / (1 - alpha)[:, None]), axis=1)
        Cp = np.sum(w, axis=0)
        eq7 = []
        for i in range(n):
            eq7.append(np.sum(g * (c[i] * T[i] - Cp) / (1 - alpha[i])))
            Cp = Cp - T[i] * alpha[i] * c[i]
        np.testing.assert_allclose(eq4, eq7, rtol=1e-10, atol=1e-12)


def test_selected_splat_gradients_match_full_backward():
    scene, cam, _ = syn.tiny_scene_1k()
    g = syn.uniform_image(cam.height, cam.width, seed=13, lo=-1.0, hi=1.0)
    full = oracle.backward(scene, cam, g)
    rng = np.random.default_rng(14)
    ids = rng.choice(scene.n, size=12, replace=False)
    sel = oracle.splat_grads(scene, cam, g, ids)
    for k in ("means", "scales", "quats", "opacities", "sh", "g2d"):
        np.testing.assert_allclose(sel[k], full[k][ids], rtol=1e-9, atol=1e-12)


def _quantize_numpy(x, fmt):
    """Reduced-precision round trip by library routines: numpy's float16
    conversion (round to nearest even), or unorm with numpy's half-to-even round."""
    x = np.asarray(x, dtype=np.float64)
    if fmt == "fp16":
        return x.astype(np.float16).astype(np.float64)
    s = 65535.0 if fmt == "unorm16" else 255.0
    return np.round(np.clip(x, 0.0, 1.0) * s) / s


def test_cprime_from_rounded_state_matches_closed_form():
    """The backward's C'_1 taken from a reduced-precision stored colour (Sec. 3.3):
    for one splat every pixel holds one fragment with T = 1, so Eq. 7 gives
    dL/dalpha = g . (c - round(C)) / (1 - alpha) against g . c when C'_1 = C; the
    opacity accumulator therefore moves by sum_p G_p g_p . (C_p - round(C_p)) /
    (1 - alpha_p), with C_p, alpha_p = 1 - T_p from the (pinned) forward and the
    rounding by numpy.  Colour gradients (Eq. 3) do not involve C'."""
    W = H = 24
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 40.0, W, H)
    sc = _one_splat((0.05, -0.03, 0.0), (0.3, 0.22, 0.26), (0.9, 0.1, -0.2, 0.3), 0.7,
                    (0.83, 0.41, 0.17))
    g = syn.uniform_image(H, W, seed=15, lo=-1.0, hi=1.0).astype(np.float64)
    for fmt in ("fp16", "unorm8"):
        ex = oracle.backward(sc, cam, g, oracle.opts_array(t_cull=0.0, clamp01=True))
        q = oracle.backward(sc, cam, g, oracle.opts_array(t_cull=0.0, clamp01=True,
                                                          quant=oracle.QUANT[fmt]),
                            quant_cprime=True)
        r = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0, clamp01=True))
        C, T, nf = r["color"], r["T"], r["nfrag"]
        alpha = 1.0 - T
        o = float(sc.opacities[0])
        m = (nf == 1) & (alpha < 0.99)
        delta = np.sum(g * (C - _quantize_numpy(C, fmt)), axis=2)   # g . (C - round(C))
        expect = np.sum((alpha[m] / o) * delta[m] / (1.0 - alpha[m]))
        got = q["g2d"][0, 8] - ex["g2d"][0, 8]
        assert abs(expect) > 1e-6
        assert abs(got - expect) <= 1e-9 * max(1.0, abs(expect)), (fmt, got, expect)
        np.testing.assert_allclose(q["g2d"][0, 5:8], ex["g2d"][0, 5:8], rtol=1e-12, atol=1e-15)
        np.testing.assert_allclose(q["sh"], ex["sh"], rtol=1e-12, atol=1e-15)


def _three_fragment_pixel():
    """Three splats straddling the optical axis at increasing depth; the pixel
    at the image centre holds one fragment of each (opacities chosen so that
    every alpha lies in (1/255, 0.99))."""
    sh = np.zeros((3, 1, 3), np.float32)
    rgbs = ((0.9, 0.2, 0.35), (0.15, 0.75, 0.6), (0.55, 0.45, 0.95))
    for i, rgb in enumerate(rgbs):
        sh[i, 0] = (np.array(rgb) - 0.5) / Y00
    sc = syn.Scene(np.array([[0.01, 0.02, -1.0], [-0.03, 0.0, 0.0], [0.02, -0.01, 1.0]], np.float32),
                   np.array([[0.4, 0.35, 0.3], [0.5, 0.5, 0.45], [0.6, 0.55, 0.6]], np.float32),
                   np.array([[1, 0, 0, 0], [0.9, 0.2, 0.1, 0.0], [0.8, 0.0, 0.3, 0.2]], np.float32),
                   np.array([0.55, 0.6, 0.85], np.float32), sh, 0)
    cam = syn.look_at((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 40.0, 9, 9)
    return sc, cam, 4 * 9 + 4


@pytest.mark.parametrize("fmt", ["fp16", "unorm16", "unorm8"])
def test_per_fragment_rounding_matches_a_hand_loop(fmt):
    """The paper's render-target round trip (Sec. 3.3): with per-fragment
    rounding the state (C, T) is rounded after every blend.  A hand-written
    loop over the three fragments of one pixel, taking the splats' projected
    alpha and colour from the oracle's projection and rounding with numpy,
    gives the same colour and transmittance; store-only rounding differs."""
    sc, cam, pix = _three_fragment_pixel()
    P = oracle.project(sc, cam, clamp01=True)
    px, py = pix % cam.width + 0.5, pix // cam.width + 0.5
    C, T = np.zeros(3), 1.0
    for i in np.argsort(P[:, 12], kind="stable"):
        dx, dy = px - P[i, 1], py - P[i, 2]
        power = -0.5 * (P[i, 6] * dx * dx + 2.0 * P[i, 7] * dx * dy + P[i, 8] * dy * dy)
        alpha = min(0.99, float(sc.opacities[i]) * math.exp(power))
        assert 1.0 / 255.0 < alpha < 0.99
        C = _quantize_numpy(C + T * alpha * P[i, 9:12], fmt)
        T = float(_quantize_numpy(T * (1.0 - alpha), fmt))
    opts = dict(t_cull=0.0, clamp01=True, quant=oracle.QUANT[fmt])
    r = oracle.render(sc, cam, oracle.opts_array(per_fragment=True, **opts), pixels=[pix])
    assert r["nfrag"][0] == 3
    np.testing.assert_allclose(r["color"][0], C, rtol=0, atol=1e-12)
    assert abs(r["T"][0] - T) <= 1e-12
    store = oracle.render(sc, cam, oracle.opts_array(**opts), pixels=[pix])
    exact = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0, clamp01=True), pixels=[pix])
    np.testing.assert_array_equal(store["color"][0], _quantize_numpy(exact["color"][0], fmt))
    if fmt == "unorm8":   # three roundings of 1/510 each: the two emulations part
        assert np.max(np.abs(r["color"][0] - store["color"][0])) > 0.0
    # without a reduced format the per-fragment mode is the exact render
    r0 = oracle.render(sc, cam, oracle.opts_array(t_cull=0.0, clamp01=True, per_fragment=True),
                       pixels=[pix])
    np.testing.assert_array_equal(r0["color"], exact["color"])


def test_torch_gradcheck_on_oracle_binding():
    """torch.autograd.gradcheck (FP64 central differences) on an autograd
    Function whose forward and backward are the oracle's."""
    torch = pytest.importorskip("torch")

    bands = dict(band_cut=1e-3, band_clamp=1e-3)
    seed = 700
    while True:
        sc, cam = _fd_scene(seed, n=5, deg=2, size=16)
        if _clean(sc, cam, oracle.opts_array(t_cull=0.0, **bands)):
            break
        seed += 1
        assert seed < 1000
    opts = oracle.opts_array(t_cull=0.0)

    class OracleRender(torch.autograd.Function):
        @staticmethod
        def forward(ctx, m, s, q, o, sh):
            ctx.save_for_backward(m, s, q, o, sh)
            scene = syn.Scene(m.numpy(), s.numpy(), q.numpy(), o.numpy(), sh.numpy(), sc.sh_degree)
            return torch.from_numpy(oracle.render(scene, cam, opts)["color"])

        @staticmethod
        def backward(ctx, g):
            m, s, q, o, sh = ctx.saved_tensors
            scene = syn.Scene(m.numpy(), s.numpy(), q.numpy(), o.numpy(), sh.numpy(), sc.sh_degree)
            r = oracle.backward(scene, cam, g.numpy(), opts)
            return tuple(torch.from_numpy(r[k]) for k in ("means", "scales", "quats", "opacities", "sh"))

    inputs = tuple(torch.tensor(a.astype(np.float64), requires_grad=True) for a in sc.arrays())
    assert torch.autograd.gradcheck(OracleRender.apply, inputs, eps=1e-6, atol=1e-6, rtol=1e-4)
