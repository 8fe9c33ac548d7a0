"""Pins of the FP64 oracle against mathematics and the paper (no GPU).

Each test checks the oracle against something other than itself: a closed
form, a conservation law, a brute-force recomputation with a different
algorithm, a textbook value, or central finite differences.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2605_13794_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _scene(n, seed, opacity_max=None, depth=(2.0, 6.0), scale=(1e-3, 5e-2)):
    rng = np.random.default_rng(seed)
    g = synth.plain_scene(n, seed)
    g.mean[:, 2] = rng.uniform(*depth, n).astype(np.float32)
    g.log_scale[:] = rng.uniform(math.log(scale[0]), math.log(scale[1]), (n, 3)).astype(np.float32)
    if opacity_max is not None:
        o = rng.uniform(0.05, opacity_max, n)
        g.opacity_logit[:] = np.log(o / (1 - o)).astype(np.float32)
    return g


# ---- spherical harmonics ------------------------------------------------

def test_sh_orthonormal_by_quadrature(oracle_mod):
    # Gauss-Legendre in cos(theta) x uniform in phi integrates degree <= 6 exactly
    z, wz = np.polynomial.legendre.leggauss(12)
    nphi = 16
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    Z, PHI = np.meshgrid(z, phi, indexing="ij")
    S = np.sqrt(1 - Z ** 2)
    dirs = np.stack([S * np.cos(PHI), S * np.sin(PHI), Z], -1).reshape(-1, 3)
    w = (wz[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    Y = oracle_mod.sh_basis(dirs)
    gram = (Y * w[:, None]).T @ Y
    assert np.abs(gram - np.eye(16)).max() < 1e-12


def test_sh_addition_theorem(oracle_mod):
    # Unsold: sum_m Y_lm(d)^2 = (2l+1)/(4 pi) for every unit d
    rng = np.random.default_rng(5)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = oracle_mod.sh_basis(d)
    for l in range(4):
        band = (Y[:, l * l:(l + 1) ** 2] ** 2).sum(1)
        assert np.allclose(band, (2 * l + 1) / (4 * np.pi), atol=1e-13)


def test_sh_textbook_values(oracle_mod):
    cases = json.load(open(os.path.join(GOLDEN, "sh_values.json")))["cases"]
    for c in cases:
        Y = oracle_mod.sh_basis(np.array(c["dir"], float))
        assert abs(Y[0, c["k"]] - c["value"]) < 1e-12, c


def test_sh_gradient_fd(oracle_mod):
    rng = np.random.default_rng(6)
    d = rng.standard_normal((20, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    _, dY = oracle_mod.sh_basis(d, with_grad=True)
    h = 1e-6
    for e in range(3):
        dp, dm = d.copy(), d.copy()
        dp[:, e] += h
        dm[:, e] -= h
        fd = (oracle_mod.sh_basis(dp) - oracle_mod.sh_basis(dm)) / (2 * h)
        assert np.abs(fd - dY[:, :, e]).max() < 1e-8


# ---- projection -----------------------------------------------------------

def _one(mean, log_s, quat, opac_logit, sh_dc=(0.0, 0.0, 0.0)):
    g = synth.GaussianSet(
        mean=np.array(mean, np.float32).reshape(1, 3), log_scale=np.array(log_s, np.float32).reshape(1, 3),
        quat=np.array(quat, np.float32).reshape(1, 4), opacity_logit=np.array([opac_logit], np.float32),
        sh=np.zeros((1, 16, 3), np.float32), lod=np.zeros(1, np.uint8))
    g.sh[0, 0, :] = np.array(sh_dc, np.float32)
    return g


@pytest.mark.parametrize("sigma,z", [(0.01, 3.0), (0.03, 2.5), (0.002, 5.0)])
def test_isotropic_on_axis_closed_form(oracle_mod, sigma, z):
    cam = synth.plain_camera(64, 64, 300.0)
    P = oracle_mod.Params()
    rng = np.random.default_rng(7)
    q = rng.standard_normal(4)
    dc = 0.3
    g = _one([0.0, 0.0, z], [math.log(sigma)] * 3, q, 0.8, (dc, dc, dc))
    g64 = oracle_mod.gaussians64(g)
    pr = oracle_mod.project(g64, cam, P)
    f = float(np.float32(300.0))
    dil = float(np.float32(0.3))
    s_stored = math.exp(float(np.float32(math.log(sigma))))  # the scale the stored log-scale encodes
    s2 = (f * s_stored / z) ** 2 + dil
    # conic of (s2) I, and the extent uses max(0.1, mid^2 - det) = 0.1 for a disc
    assert pr["status"][0] == oracle_mod.ACTIVE
    assert np.allclose(pr["conic"][0], [1 / s2, 0.0, 1 / s2], rtol=1e-12, atol=1e-12)
    assert pr["radius"][0] == math.ceil(3 * math.sqrt(s2 + math.sqrt(0.1)))
    assert np.allclose(pr["uv"][0], [32.0, 32.0])
    # image: alpha(rho) c at every pixel, zero below alpha_min, one Gaussian never stops early
    fwd = oracle_mod.forward_view(g64, cam, P)
    o = 1 / (1 + math.exp(-float(np.float32(0.8))))
    c = float(np.float32(dc)) * 0.28209479177387814 + 0.5
    ys, xs = np.mgrid[0:64, 0:64] + 0.5
    rho2 = (xs - 32.0) ** 2 + (ys - 32.0) ** 2
    alpha = np.minimum(float(np.float32(0.99)), o * np.exp(-0.5 * rho2 / s2))
    alpha[alpha < float(np.float32(1 / 255))] = 0.0
    r = pr["radius"][0]
    # pixels whose tile lies outside the footprint rectangle receive nothing
    rect = pr["rect"][0]
    tx, ty = (xs // 16).astype(int), (ys // 16).astype(int)
    inside = (tx >= rect[0]) & (tx < rect[2]) & (ty >= rect[1]) & (ty < rect[3])
    alpha[~inside] = 0.0
    assert r > 0
    np.testing.assert_allclose(fwd["image"][0], alpha * c, atol=1e-12)
    np.testing.assert_allclose(fwd["T"], 1 - alpha, atol=1e-12)
    # importance of the single Gaussian: w = sum alpha T (T = 1), a = pixels with alpha >= alpha_min
    assert abs(fwd["w"][0] - alpha.sum()) < 1e-10
    assert fwd["a"][0] == np.count_nonzero(alpha)


def test_lod_gate_table(oracle_mod):
    gold = json.load(open(os.path.join(GOLDEN, "lod_gate.json")))
    cam = synth.plain_camera(64, 64, 300.0)
    P = oracle_mod.Params(lod_enable=True, lod_d0=gold["d0"], lod_f=gold["f"], lod_Lmax=gold["Lmax"])
    for d, L in gold["cases"]:
        for lod in range(7):
            g = _one([0.0, 0.0, d], [0.0] * 3, [1, 0, 0, 0], 0.0)
            g.lod[0] = lod
            pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P)
            gated = pr["status"][0] == oracle_mod.GATED_LOD
            assert gated == (lod > L), (d, lod, L)


def test_near_plane_and_cull_mask(oracle_mod):
    cam = synth.plain_camera(64, 64, 300.0)
    P = oracle_mod.Params(cull_enable=True)
    g = _one([0.0, 0.0, 0.1], [math.log(0.01)] * 3, [1, 0, 0, 0], 0.0)
    assert oracle_mod.project(oracle_mod.gaussians64(g), cam, P)["status"][0] == oracle_mod.NEAR
    g = _one([0.0, 0.0, 3.0], [math.log(0.01)] * 3, [1, 0, 0, 0], 0.0)
    pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P, cull=np.array([1], np.uint32))
    assert pr["status"][0] == oracle_mod.GATED_CULL
    pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P, cull=np.array([0], np.uint32))
    assert pr["status"][0] == oracle_mod.ACTIVE


# ---- compositing --------------------------------------------------------

def test_two_gaussians_by_hand(oracle_mod):
    # two tiny Gaussians centred on the same pixel centre; the nearer composites first
    cam = synth.plain_camera(16, 16, 300.0)
    cam.cx = cam.cy = 8.5  # pixel (8, 8) centre on the optical axis
    P = oracle_mod.Params()
    ls = math.log(1e-4)
    g = _one([0.0, 0.0, 3.0], [ls] * 3, [1, 0, 0, 0], math.log(0.6 / 0.4), (1.0, 0.0, 0.0))
    g2 = _one([0.0, 0.0, 2.0], [ls] * 3, [1, 0, 0, 0], math.log(0.5 / 0.5), (0.0, 1.0, 0.0))
    both = synth.GaussianSet(*[np.concatenate([getattr(g, k), getattr(g2, k)], axis=0)
                               for k in ("mean", "log_scale", "quat", "opacity_logit", "sh", "lod")])
    fwd = oracle_mod.forward_view(oracle_mod.gaussians64(both), cam, P)
    C0 = 0.28209479177387814
    o1 = 1 / (1 + math.exp(-float(np.float32(math.log(0.6 / 0.4)))))
    o2 = 0.5
    c1 = np.array([C0 + 0.5, 0.5, 0.5])
    c2 = np.array([0.5, C0 + 0.5, 0.5])
    # at the centre the dilated footprint peaks at exp(0) = 1, so alpha = opacity
    expect = o2 * c2 + (1 - o2) * o1 * c1
    np.testing.assert_allclose(fwd["image"][:, 8, 8], expect, atol=1e-12)
    assert abs(fwd["T"][8, 8] - (1 - o1) * (1 - o2)) < 1e-12
    assert fwd["n_contrib"][8, 8] == 2
    # tile list order: Gaussian 1 (nearer) before Gaussian 0
    ts, lst = fwd["bins"]
    assert list(lst[ts[0]:ts[1]]) == [1, 0]


def _pixel_case(oracle_mod, frags):
    """Composites pixel (0, 0) over explicit fragments (offset d from the pixel
    centre along x, opacity) with a unit isotropic conic: power = -d^2 / 2."""
    n = len(frags)
    proj = dict(uv=np.array([[0.5 + d, 0.5] for d, _ in frags]), conic=np.tile([1.0, 0.0, 1.0], (n, 1)),
                opacity=np.array([o for _, o in frags]), rgb=np.full((n, 3), 0.5))
    return oracle_mod.render_pixels(proj, [[0, 0]], [list(range(n))], oracle_mod.Params())


def _offset_for(alpha, o):
    return math.sqrt(-2.0 * math.log(alpha / o))


def test_threshold_flags(oracle_mod):
    # a fragment within rounding of a threshold flags its pixel; one a percent away does not
    O, P = oracle_mod, oracle_mod.Params()
    # the thresholds as the renderer holds them: FP32
    amin, amax, tmin = (float(np.float32(x)) for x in (P.alpha_min, P.alpha_max, P.T_min))
    near = _pixel_case(O, [(_offset_for(amin * (1 + 1e-7), 0.5), 0.5)])
    assert near["flags"][0] & O.PIX_ALPHA_MIN and near["n_contrib"][0] == 1
    far = _pixel_case(O, [(_offset_for(amin * 1.01, 0.5), 0.5)])
    assert far["flags"][0] == 0
    below = _pixel_case(O, [(_offset_for(amin * (1 - 1e-7), 0.5), 0.5)])
    assert below["flags"][0] & O.PIX_ALPHA_MIN and below["n_contrib"][0] == 0
    assert _pixel_case(O, [(0.0, amax * (1 - 1e-7))])["flags"][0] & O.PIX_ALPHA_MAX
    assert _pixel_case(O, [(0.0, amax * 0.98)])["flags"][0] == 0
    # T_min: 1 - 0.99 leaves T = 0.01; the second fragment lands T(1 - alpha) next to T_min
    a2 = 1.0 - tmin * (1 + 1e-7) / (1.0 - amax)
    t_near = _pixel_case(O, [(0.0, 0.999), (0.0, a2)])
    assert t_near["flags"][0] & O.PIX_T_MIN and t_near["n_contrib"][0] == 2
    t_far = _pixel_case(O, [(0.0, 0.999), (0.0, 0.9)])
    assert t_far["flags"][0] == 0
    # flags never change what is composited
    np.testing.assert_allclose(near["T"][0], 1.0 - amin * (1 + 1e-7), rtol=1e-12)


def test_equal_depth_ties_by_index(oracle_mod):
    cam = synth.plain_camera(16, 16, 300.0)
    P = oracle_mod.Params()
    g = synth.plain_scene(6, 11)
    g.mean[:] = np.array([[0.0, 0.0, 3.0]], np.float32)
    g.log_scale[:] = np.float32(math.log(0.01))
    fwd = oracle_mod.forward_view(oracle_mod.gaussians64(g), cam, P)
    ts, lst = fwd["bins"]
    assert list(lst[ts[0]:ts[1]]) == sorted(lst[ts[0]:ts[1]])


def test_transmittance_invariant(oracle_mod):
    # all colours 1 and bg 0: C(p) = sum alpha_i T_i = 1 - T_final (telescoping product)
    g = synth.plain_scene(3000, 21)
    g.sh[:] = 0.0
    g.sh[:, 0, :] = np.float32(0.5 / 0.28209479177387814)
    cam = synth.plain_camera(96, 80, 200.0)
    P = oracle_mod.Params()
    fwd = oracle_mod.forward_view(oracle_mod.gaussians64(g), cam, P)
    assert fwd["T"].min() < 0.01  # the test covers saturated pixels
    for c in range(3):
        np.testing.assert_allclose(fwd["image"][c], 1.0 - fwd["T"], atol=1e-6)
    # importance: sum_i w_i = sum_p (1 - T_final)
    assert abs(fwd["w"].sum() - (1 - fwd["T"]).sum()) < 1e-8 * fwd["T"].size


def test_bg_colour_enters_through_final_transmittance(oracle_mod):
    g = synth.plain_scene(2000, 22)
    cam = synth.plain_camera(64, 64, 200.0)
    P0 = oracle_mod.Params()
    P1 = oracle_mod.Params(bg=(0.25, 0.5, 1.0))
    g64 = oracle_mod.gaussians64(g)
    f0 = oracle_mod.forward_view(g64, cam, P0)
    f1 = oracle_mod.forward_view(g64, cam, P1)
    bg = np.array([np.float32(0.25), np.float32(0.5), np.float32(1.0)], float)
    np.testing.assert_allclose(f1["image"], f0["image"] + bg[:, None, None] * f0["T"][None], atol=1e-12)


TILE_SHAPES = [(16, 16), (32, 8), (8, 32), (32, 16), (16, 8), (8, 16)]


@pytest.mark.parametrize("tw,th", TILE_SHAPES)
def test_tiled_equals_untiled_brute_force(oracle_mod, tw, th):
    # With opacity below alpha_min * e^{4.5} = 0.35 every fragment outside a
    # Gaussian's 3-sigma rectangle has alpha < alpha_min, so compositing all
    # Gaussians at every pixel (no tiles, no rectangles) must give the same
    # image, whatever the tile shape.
    g = _scene(1500, 23, opacity_max=0.34)
    cam = synth.plain_camera(80, 64, 250.0)
    P = oracle_mod.Params(tile_w=tw, tile_h=th)
    g64 = oracle_mod.gaussians64(g)
    fwd = oracle_mod.forward_view(g64, cam, P)
    img, T = oracle_mod.render_brute(fwd["proj"], cam, P)
    assert np.array_equal(img, fwd["image"])
    assert np.array_equal(T, fwd["T"])


@pytest.mark.parametrize("tw,th", TILE_SHAPES)
def test_rect_is_the_tiles_meeting_the_3sigma_box(oracle_mod, tw, th):
    # the rectangle holds exactly the tiles whose pixel span meets
    # [u - r, u + r] x [v - r, v + r], clipped to the image
    g = synth.plain_scene(600, 27)
    cam = synth.plain_camera(100, 70, 250.0)
    P = oracle_mod.Params(tile_w=tw, tile_h=th)
    pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P)
    tx, ty = oracle_mod.tiles_of(cam, P)
    act = np.nonzero(pr["status"] == oracle_mod.ACTIVE)[0]
    assert len(act) > 100
    for i in act:
        u, v = pr["uv"][i]
        r = pr["radius"][i]
        xs = [x for x in range(tx) if x * tw <= u + r and u - r < (x + 1) * tw]
        ys = [y for y in range(ty) if y * th <= v + r and v - r < (y + 1) * th]
        x0, y0, x1, y1 = pr["rect"][i]
        assert (list(range(x0, x1)), list(range(y0, y1))) == (xs, ys), i


def test_binning_brute_force(oracle_mod):
    g = synth.plain_scene(800, 24)
    cam = synth.plain_camera(100, 70, 250.0)
    P = oracle_mod.Params()
    pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P)
    ts, lst = oracle_mod.bin_tiles(pr, cam, P)
    tx, ty = oracle_mod.tiles_of(cam, P)
    for t in range(tx * ty):
        x, y = t % tx, t // tx
        members = [i for i in range(g.n) if pr["status"][i] == oracle_mod.ACTIVE and
                   pr["rect"][i, 0] <= x < pr["rect"][i, 2] and pr["rect"][i, 1] <= y < pr["rect"][i, 3]]
        members.sort(key=lambda i: (pr["depth32"][i].view(np.uint32), i))
        assert list(lst[ts[t]:ts[t + 1]]) == members


# ---- backward: central finite differences of the FP64 forward -------------

def _loss_and_state(oracle_mod, g64, cam, P, dL):
    f = oracle_mod.forward_view(g64, cam, P)
    state = (f["proj"]["status"].tobytes(), f["proj"]["rect"].tobytes(), f["n_contrib"].tobytes(),
             f["proj"]["clamp"].tobytes())
    return float((f["image"] * dL).sum()), state, f


@pytest.mark.parametrize("seed", [31, 32])
def test_backward_matches_central_differences(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    g = _scene(14, seed, opacity_max=0.9, depth=(2.0, 3.0), scale=(0.01, 0.04))
    g.mean[:, 0] = rng.uniform(-0.25, 0.25, g.n).astype(np.float32)
    g.mean[:, 1] = rng.uniform(-0.25, 0.25, g.n).astype(np.float32)
    cam = synth.plain_camera(48, 40, 120.0)
    P = oracle_mod.Params()
    g64 = oracle_mod.gaussians64(g)
    dL = rng.standard_normal((3, cam.height, cam.width))
    L0, st0, f0 = _loss_and_state(oracle_mod, g64, cam, P, dL)
    assert (f0["proj"]["status"] == oracle_mod.ACTIVE).all()
    grads = oracle_mod.backward_view(g64, f0, cam, P, dL)
    checked = 0
    for name in ("mean", "log_scale", "quat", "opacity_logit", "sh"):
        arr = g64[name]
        flat = arr.reshape(-1)
        gflat = grads[name].reshape(-1)
        idx = range(flat.size) if name != "sh" else rng.choice(flat.size, 120, replace=False)
        for k in idx:
            x0 = flat[k]
            h = 1e-6 * max(1.0, abs(x0))
            flat[k] = x0 + h
            Lp, stp, _ = _loss_and_state(oracle_mod, g64, cam, P, dL)
            flat[k] = x0 - h
            Lm, stm, _ = _loss_and_state(oracle_mod, g64, cam, P, dL)
            flat[k] = x0
            if stp != st0 or stm != st0:
                continue  # a discrete decision moved: the derivative is not defined there
            fd = (Lp - Lm) / (2 * h)
            assert abs(fd - gflat[k]) <= 1e-5 * max(1.0, abs(fd)), (name, k, fd, gflat[k])
            checked += 1
    assert checked > 0.9 * (g.n * (3 + 3 + 4 + 1) + 120)


# ---- importance selection -----------------------------------------------------

def test_visible_set_is_minimal_by_exhaustion(oracle_mod):
    rng = np.random.default_rng(41)
    for trial in range(40):
        n = 9
        w = rng.choice([0.0, 0.5, 1.0, 2.0, rng.uniform(0, 3)], size=n) if trial % 2 else rng.uniform(0, 1, n)
        total = w.sum()
        vis = oracle_mod.visible_top_mass(w, 0.99)
        if total == 0:
            assert not vis.any()
            continue
        # smallest cardinality of any subset carrying 99 %
        best = min(bin(m).count("1") for m in range(1 << n)
                   if sum(w[i] for i in range(n) if m >> i & 1) >= 0.99 * total)
        assert vis.sum() == best
        assert w[vis].sum() >= 0.99 * total
        # the chosen members are the largest w, ties resolved toward lower index
        order = sorted(range(n), key=lambda i: (-w[i], i))
        assert set(np.nonzero(vis)[0]) == set(order[:best])


# ---- loss and optimizer -----------------------------------------------------------

def test_ssim_identity_and_gradient(oracle_mod):
    rng = np.random.default_rng(51)
    x = rng.uniform(0, 1, (3, 20, 24))
    s, gs = oracle_mod.ssim_and_grad(x, x)
    assert abs(s - 1.0) < 1e-12 and np.abs(gs).max() < 1e-12
    y = rng.uniform(0, 1, (3, 20, 24))
    s, gs = oracle_mod.ssim_and_grad(x, y)
    h = 1e-6
    for _ in range(25):
        idx = tuple(rng.integers(0, d) for d in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle_mod.ssim_and_grad(xp, y)[0] - oracle_mod.ssim_and_grad(xm, y)[0]) / (2 * h)
        assert abs(fd - gs[idx]) < 1e-7


def test_photometric_loss_gradient(oracle_mod):
    rng = np.random.default_rng(52)
    x = rng.uniform(0, 1, (2, 3, 16, 18))
    y = rng.uniform(0, 1, (2, 3, 16, 18))
    L, g = oracle_mod.photometric_loss(x, y)
    L0, _ = oracle_mod.photometric_loss(y, y)
    assert abs(L0) < 1e-12
    h = 1e-6
    for _ in range(20):
        idx = tuple(rng.integers(0, d) for d in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (oracle_mod.photometric_loss(xp, y)[0] - oracle_mod.photometric_loss(xm, y)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-7


def test_scale_regulariser(oracle_mod):
    ls = np.log(np.array([[0.1, 0.5, 2.0], [0.2, 0.05, 3.0], [0.3, 0.6, 0.7]]))
    vis = np.array([True, True, False])
    val, g = oracle_mod.scale_regulariser(ls, vis, beta=10.0)
    assert abs(val - 10.0 * (0.1 + 0.05) / 2) < 1e-12
    h = 1e-7
    for idx in np.ndindex(ls.shape):
        lp, lm = ls.copy(), ls.copy()
        lp[idx] += h
        lm[idx] -= h
        fd = (oracle_mod.scale_regulariser(lp, vis)[0] - oracle_mod.scale_regulariser(lm, vis)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6


def test_adam_first_step_closed_form(oracle_mod):
    rng = np.random.default_rng(53)
    p = rng.standard_normal(100)
    g = rng.standard_normal(100)
    z = np.zeros(100)
    p1, m1, v1 = oracle_mod.adam_step(p, g, z, z, step=1, lr=0.01, eps=1e-15)
    # bias-corrected moments equal g and g^2 after one step
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-15), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_ssim_value_against_library_gaussian_filter(oracle_mod):
    # the local statistics from scipy's Gaussian filter (sigma 1.5, radius 5, zero
    # padding, one image plane at a time) put into the SSIM index of Wang et al.
    # (2004); pins the oracle's window, its normalisation and its padding
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(54)
    x = rng.uniform(0, 1, (3, 19, 23))
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1)

    def blur(a):
        return ndimage.gaussian_filter(a, sigma=(0, 1.5, 1.5), truncate=5 / 1.5, mode="constant", cval=0.0)

    C1, C2 = 0.01 ** 2, 0.03 ** 2
    mx, my = blur(x), blur(y)
    vx, vy, cxy = blur(x * x) - mx ** 2, blur(y * y) - my ** 2, blur(x * y) - mx * my
    ref = ((2 * mx * my + C1) * (2 * cxy + C2) / ((mx ** 2 + my ** 2 + C1) * (vx + vy + C2))).mean()
    s, _ = oracle_mod.ssim_and_grad(x, y)
    assert abs(s - ref) < 1e-12
    assert s < 0.9  # a real difference, not the identity


def test_adam_constant_gradient_closed_form(oracle_mod):
    # with a constant gradient from zero moments the bias-corrected moments are
    # g and g^2 at every step, so each step moves p by lr * g / (|g| + eps)
    rng = np.random.default_rng(55)
    p0 = rng.standard_normal(64)
    g = rng.standard_normal(64)
    b1, b2, lr, eps = 0.9, 0.999, 0.01, 1e-15
    p, m, v = p0, np.zeros(64), np.zeros(64)
    for t in range(1, 51):
        p, m, v = oracle_mod.adam_step(p, g, m, v, step=t, lr=lr, beta1=b1, beta2=b2, eps=eps)
        np.testing.assert_allclose(m, (1 - b1 ** t) * g, rtol=1e-12, atol=0)
        np.testing.assert_allclose(v, (1 - b2 ** t) * g * g, rtol=1e-12, atol=0)
        np.testing.assert_allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-12)


def test_adam_zero_gradient_step_closed_form(oracle_mod):
    # a gradient step then a zero-gradient step (the step a deferred Gaussian
    # replays): m = b1 (1 - b1) g, v = b2 (1 - b2) g^2, and the bias-corrected
    # ratio is (b1 / (1 + b1)) g / sqrt(b2 / (1 + b2)) |g|
    rng = np.random.default_rng(56)
    p0 = rng.standard_normal(64)
    g = rng.standard_normal(64)
    b1, b2, lr, eps = 0.9, 0.999, 0.01, 1e-15
    z = np.zeros(64)
    p1, m1, v1 = oracle_mod.adam_step(p0, g, z, z, step=1, lr=lr, beta1=b1, beta2=b2, eps=eps)
    p2, m2, v2 = oracle_mod.adam_step(p1, z, m1, v1, step=2, lr=lr, beta1=b1, beta2=b2, eps=eps)
    np.testing.assert_allclose(m2, b1 * (1 - b1) * g, rtol=1e-12, atol=0)
    np.testing.assert_allclose(v2, b2 * (1 - b2) * g * g, rtol=1e-12, atol=0)
    step2 = lr * (b1 / (1 + b1)) * g / (np.sqrt(b2 / (1 + b2)) * np.abs(g) + eps)
    np.testing.assert_allclose(p2, p1 - step2, rtol=0, atol=1e-12)


def test_photometric_loss_weights_eq4(oracle_mod):
    # Eq. 4 with lambda = 0.2 on a target offset by a constant c: the L1 term is |c|
    # exactly, the D-SSIM term is 1 - SSIM; a batch of two copies of the view has
    # the loss of one view (mean over views)
    rng = np.random.default_rng(57)
    x = rng.uniform(0.2, 0.8, (3, 17, 21))
    c = 0.05
    y = x + c
    s, _ = oracle_mod.ssim_and_grad(x, y)
    L1, _ = oracle_mod.photometric_loss(x[None], y[None], lam=0.2)
    assert abs(L1 - (0.8 * c + 0.2 * (1.0 - s))) < 1e-12
    L2, g2 = oracle_mod.photometric_loss(np.stack([x, x]), np.stack([y, y]), lam=0.2)
    _, g1 = oracle_mod.photometric_loss(x[None], y[None], lam=0.2)
    assert abs(L2 - L1) < 1e-12
    np.testing.assert_allclose(g2[0], g1[0] / 2, rtol=1e-12, atol=1e-18)


def test_importance_accumulation_by_hand(oracle_mod):
    # Sec. 3.2 over two views of four Gaussians, worked by hand: s += w / (a + eps)
    # where a > 0, c^rad counts the views in which the Gaussian has a record, and
    # c^vis the views in whose top 99 % of w mass it lies
    O = oracle_mod
    acc = O.new_importance(4)
    st = lambda *v: {"status": np.array(v)}
    # view 1: w = (6, 3, 1, 0), masses 6, 9, 10 of 10: the 99 % cut needs all three
    v1 = O.importance_update(acc, [6.0, 3.0, 1.0, 0.0], [3, 2, 1, 0],
                             st(O.ACTIVE, O.ACTIVE, O.ACTIVE, O.GATED_LOD), eps=0.0)
    # view 2: w = (0, 200, 1, 0.5): 200 of 201.5 is 99.26 % >= 99 %, so only Gaussian 1
    v2 = O.importance_update(acc, [0.0, 200.0, 1.0, 0.5], [0, 8, 2, 1],
                             st(O.NEAR, O.ACTIVE, O.ACTIVE, O.ACTIVE), eps=0.0)
    np.testing.assert_array_equal(v1["cvis"], [True, True, True, False])
    np.testing.assert_array_equal(v2["cvis"], [False, True, False, False])
    np.testing.assert_array_equal(v2["cull"], [True, False, True, True])
    np.testing.assert_allclose(acc["s"], [6 / 3, 3 / 2 + 200 / 8, 1 / 1 + 1 / 2, 0.5 / 1], rtol=1e-15)
    np.testing.assert_array_equal(acc["crad"], [1, 2, 2, 1])
    np.testing.assert_array_equal(acc["cvis"], [1, 2, 1, 0])


def test_rotated_anisotropic_on_axis_closed_form(oracle_mod):
    # a needle rotated by 40 degrees about the optical axis, on the axis: the
    # screen covariance is (f/z)^2 R2 diag(s1^2, s2^2) R2^T + 0.3 I with R2 the
    # in-plane rotation, whose angle comes from the quaternion's half-angle
    # identities; its major axis turns from +u toward +v, so the covariance of
    # (u, v) is positive and the conic's B negative
    cam = synth.plain_camera(64, 64, 300.0)
    P = oracle_mod.Params()
    z = 3.0
    half = math.radians(20.0)
    q = [math.cos(half), 0.0, 0.0, math.sin(half)]
    ls = [math.log(0.02), math.log(0.005), math.log(0.001)]
    g = _one([0.0, 0.0, z], ls, q, 0.8)
    pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P)
    qf = np.array(q, np.float32).astype(np.float64)
    qf /= np.linalg.norm(qf)
    c, s = qf[0] ** 2 - qf[3] ** 2, 2.0 * qf[0] * qf[3]
    s1, s2 = (math.exp(float(np.float32(v))) for v in ls[:2])
    k = (float(np.float32(300.0)) / z) ** 2
    dil = float(np.float32(0.3))
    a = k * (s1 * s1 * c * c + s2 * s2 * s * s) + dil
    b = k * (s1 * s1 - s2 * s2) * s * c
    cc = k * (s1 * s1 * s * s + s2 * s2 * c * c) + dil
    det = a * cc - b * b
    assert pr["status"][0] == oracle_mod.ACTIVE
    np.testing.assert_allclose(pr["conic"][0], [cc / det, -b / det, a / det], rtol=1e-10, atol=0)
    assert b > 0 and pr["conic"][0][1] < 0
    np.testing.assert_allclose(pr["uv"][0], [32.0, 32.0])


def test_isotropic_off_axis_jacobian_term(oracle_mod):
    # an isotropic Gaussian off the axis at (x, 0, z), inside the Jacobian's
    # clamp: J = (f/z) [[1, 0, -x/z], [0, 1, 0]] stretches the u variance by
    # 1 + (x/z)^2 and leaves v and the covariance as they are
    cam = synth.plain_camera(64, 64, 300.0)
    P = oracle_mod.Params()
    sigma = 0.02
    g = _one([0.3, 0.0, 3.0], [math.log(sigma)] * 3, [1.0, 0.0, 0.0, 0.0], 0.8)
    pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P)
    x, z = float(np.float32(0.3)), 3.0
    f = float(np.float32(300.0))
    s = math.exp(float(np.float32(math.log(sigma))))
    dil = float(np.float32(0.3))
    a = (f * s / z) ** 2 * (1.0 + (x / z) ** 2) + dil
    c = (f * s / z) ** 2 + dil
    assert pr["status"][0] == oracle_mod.ACTIVE
    np.testing.assert_allclose(pr["conic"][0], [1.0 / a, 0.0, 1.0 / c], rtol=1e-10, atol=1e-15)
    np.testing.assert_allclose(pr["uv"][0], [f * x / z + 32.0, 32.0], rtol=1e-12)


def test_jacobian_clamp_beyond_the_field_of_view(oracle_mod):
    # past 1.3 tan(fov/2) the Jacobian takes the clamped ratio (the mean does
    # not): a wide Gaussian at x/z = 0.2 whose footprint reaches back into a
    # 64-pixel image with f = 300 (limit 1.3 * 32 / 300)
    cam = synth.plain_camera(64, 64, 300.0)
    P = oracle_mod.Params()
    sigma = 0.2
    g = _one([0.6, 0.0, 3.0], [math.log(sigma)] * 3, [1.0, 0.0, 0.0, 0.0], 0.8)
    pr = oracle_mod.project(oracle_mod.gaussians64(g), cam, P)
    f = float(np.float32(300.0))
    s = math.exp(float(np.float32(math.log(sigma))))
    lim = 1.3 * 32.0 / f
    a = (f * s / 3.0) ** 2 * (1.0 + lim * lim) + 0.3
    c = (f * s / 3.0) ** 2 + 0.3
    assert pr["status"][0] == oracle_mod.ACTIVE
    np.testing.assert_allclose(pr["conic"][0], [1.0 / a, 0.0, 1.0 / c], rtol=1e-6, atol=1e-12)
    assert pr["uv"][0][0] > 64.0  # the mean itself is off the image


def test_stop_before_the_fragment_that_would_pass_t_min(oracle_mod):
    # four layers of alpha 0.95 at the pixel centre: T runs 1, 0.05, 0.0025,
    # 1.25e-4; the fourth would leave 6.25e-6 < 1e-4, so the pixel stops before
    # it: three fragments composited, C = 0.5 (1 - T_final) with unit-half colours
    res = oracle_mod.render_pixels(
        dict(uv=np.full((4, 2), 0.5), conic=np.tile([1.0, 0.0, 1.0], (4, 1)), opacity=np.full(4, 0.95),
             rgb=np.full((4, 3), 0.5)), [[0, 0]], [[0, 1, 2, 3]], oracle_mod.Params())
    assert res["n_contrib"][0] == 3 and res["flags"][0] == 0
    assert abs(res["T"][0] - 0.05 ** 3) < 1e-15
    np.testing.assert_allclose(res["C"][0], 0.5 * (1.0 - 0.05 ** 3), rtol=1e-12)


def test_sh_colour_clamp_blocks_its_gradient(oracle_mod):
    # rgb = max(SH + 0.5, 0): a channel whose DC term drives it below zero is
    # black in the image and passes no gradient to any of its 16 coefficients
    cam = synth.plain_camera(32, 32, 300.0)
    P = oracle_mod.Params()
    g = _one([0.0, 0.0, 3.0], [math.log(0.01)] * 3, [1.0, 0.0, 0.0, 0.0], 0.8, (0.3, -3.0, 0.0))
    g64 = oracle_mod.gaussians64(g)
    fwd = oracle_mod.forward_view(g64, cam, P)
    assert fwd["image"][0].max() > 0.1 and fwd["image"][1].max() == 0.0
    np.testing.assert_allclose(fwd["image"][2].max() / fwd["image"][0].max(),
                               0.5 / (0.28209479177387814 * float(np.float32(0.3)) + 0.5), rtol=1e-12)
    grads = oracle_mod.backward_view(g64, fwd, cam, P, np.ones((3, cam.height, cam.width)))
    sh = grads["sh"].reshape(16, 3) if grads["sh"].size == 48 else grads["sh"][0]
    assert np.all(sh[:, 1] == 0.0)
    assert sh[0, 0] > 0.0 and sh[0, 2] > 0.0


def test_visible_set_breaks_ties_by_lower_index(oracle_mod):
    # w = (2, 3, 3, 1): the descending order with ties by index is 1, 2, 0, 3
    # (masses 3, 6, 8, 9 of 9); a cut at 30 % takes Gaussian 1 alone, at 60 %
    # Gaussians 1 and 2, at 85 % all but 3; zero mass makes nothing visible
    w = [2.0, 3.0, 3.0, 1.0]
    np.testing.assert_array_equal(oracle_mod.visible_top_mass(w, 0.3), [False, True, False, False])
    np.testing.assert_array_equal(oracle_mod.visible_top_mass(w, 0.6), [False, True, True, False])
    np.testing.assert_array_equal(oracle_mod.visible_top_mass(w, 0.85), [True, True, True, False])
    np.testing.assert_array_equal(oracle_mod.visible_top_mass([0.0, 0.0], 0.99), [False, False])
