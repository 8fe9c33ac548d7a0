"""Pins of the oracle's decision flags (no GPU).

The oracle takes every decision in FP64 and flags those an FP32 renderer may
take the other way.  These tests check the flags against independent FP32
evaluations written here with numpy float32 arithmetic:

* compositing: a renderer within the stated precision (mean within prec_mean
  pixels, exponent-form coefficients within prec_conic), perturbed to the
  limits of that precision, takes every unflagged alpha_min / alpha_max /
  T_min decision as the oracle does;
* projection: FP32 evaluations of the radius by the two standard ways of
  forming Sigma' stay within the oracle's error bound of the FP64 extent, and
  give the oracle's radius wherever it is not flagged;
* the per-Gaussian count of flagged pixels (gcount) on a case counted by hand,
  and the LOD and radius flags on constructed boundary cases.
"""
import math

import numpy as np
import pytest

from paper_2605_13794_gb300 import synth

F = np.float32


# ---- compositing ---------------------------------------------------------------

def _fp32_composite(O, fwd, cam, P, rng, scale=1.0):
    """A renderer at the limits of the stated precision: every Gaussian's mean
    moved by +-prec_mean, A and D scaled by (1 +- prec_conic), k moved by
    +-prec_conic (|k| + sqrt(D / A)) (signs drawn per Gaussian, times `scale`),
    then the exponent, alpha, transmittance and the three threshold tests in
    float32.  Returns per pixel the composited entry positions (a bitmask as
    a Python int) and n_contrib."""
    pr = fwd["proj"]
    ts, lst = fwd["bins"]
    n = pr["status"].shape[0]
    A, B, C = pr["conic"][:, 0], pr["conic"][:, 1], pr["conic"][:, 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        k = np.where(A > 0, B / A, 0.0)
        D = C - B * k
        kb = np.abs(k) + np.sqrt(np.where(A > 0, np.abs(D / A), 0.0))
    sg = lambda: rng.choice([-1.0, 1.0], n) * scale
    A32 = F(A * (1 + sg() * P.prec_conic))
    D32 = F(D * (1 + sg() * P.prec_conic))
    k32 = F(k + sg() * P.prec_conic * kb)
    u32 = pr["uv"][:, 0] + sg() * P.prec_mean
    v32 = pr["uv"][:, 1] + sg() * P.prec_mean
    o32 = F(pr["opacity"])
    amin, amax, tmin = F(P.alpha_min), F(P.alpha_max), F(P.T_min)
    W, H = cam.width, cam.height
    tiles_x = (W + P.tile_w - 1) // P.tile_w
    comp = np.zeros((H, W), object)
    ncon = np.zeros((H, W), np.int64)
    for t in range(len(ts) - 1):
        ty, tx = divmod(t, tiles_x)
        ys, xs = np.mgrid[ty * P.tile_h:min((ty + 1) * P.tile_h, H), tx * P.tile_w:min((tx + 1) * P.tile_w, W)]
        ys, xs = ys.ravel(), xs.ravel()
        T = np.ones(len(xs), F)
        done = np.zeros(len(xs), bool)
        nc = np.zeros(len(xs), np.int64)
        bits = [0] * len(xs)
        for j, g in enumerate(lst[ts[t]:ts[t + 1]]):
            # pixel offsets from the mean, rounded to float32 (the mean held in double)
            dx = F(xs + 0.5 - u32[g])
            dy = F(ys + 0.5 - v32[g])
            e = F(dx + F(k32[g] * dy))
            p = F(F(-0.5) * F(F(A32[g] * F(e * e)) + F(F(D32[g] * dy) * dy)))
            al = np.minimum(amax, F(o32[g] * np.exp(p).astype(F)))
            ok = ~done & (p <= 0) & (al >= amin)
            tT = F(T * F(F(1) - al))
            stop = ok & (tT < tmin)
            c = ok & ~stop
            done |= stop
            T = np.where(c, tT, T)
            nc = np.where(c, j + 1, nc)
            for q in np.nonzero(c)[0]:
                bits[q] |= 1 << j
        for q in range(len(xs)):
            comp[ys[q], xs[q]] = bits[q]
            ncon[ys[q], xs[q]] = nc[q]
    return comp, ncon


@pytest.mark.parametrize("seed", [61, 62])
def test_compositing_flags_cover_an_fp32_renderer(oracle_mod, seed):
    O = oracle_mod
    g = synth.plain_scene(3000, seed=seed)
    cam = synth.plain_camera(96, 80, 140.0)
    P = O.Params(bg=(0.1, 0.2, 0.3))
    fwd = O.forward_view(O.gaussians64(g), cam, P)
    ok = fwd["flags"] == 0
    assert ok.mean() > 0.99
    # the oracle's own composited sets, from its FP64 walk
    ref_comp, ref_nc = _fp32_composite_ref(O, fwd, cam, P)
    assert np.array_equal(ref_nc, fwd["n_contrib"])
    rng = np.random.default_rng(seed + 1)
    for _ in range(3):
        comp, nc = _fp32_composite(O, fwd, cam, P, rng)
        assert np.array_equal(nc[ok], fwd["n_contrib"][ok])
        assert all(comp[y, x] == ref_comp[y, x] for y, x in zip(*np.nonzero(ok)))
    # the emulation is sensitive: forty times the stated precision flips some
    # unflagged decision (so the agreement above is not vacuous)
    flips = 0
    for _ in range(3):
        comp, nc = _fp32_composite(O, fwd, cam, P, rng, scale=40.0)
        flips += sum(comp[y, x] != ref_comp[y, x] for y, x in zip(*np.nonzero(ok)))
    assert flips > 0


def _fp32_composite_ref(O, fwd, cam, P):
    """The same walk in FP64 without perturbation: the oracle's decisions."""
    pr = fwd["proj"]
    ts, lst = fwd["bins"]
    W, H = cam.width, cam.height
    tiles_x = (W + P.tile_w - 1) // P.tile_w
    amin, amax, tmin = float(F(P.alpha_min)), float(F(P.alpha_max)), float(F(P.T_min))
    comp = np.zeros((H, W), object)
    ncon = np.zeros((H, W), np.int64)
    for t in range(len(ts) - 1):
        ty, tx = divmod(t, tiles_x)
        ys, xs = np.mgrid[ty * P.tile_h:min((ty + 1) * P.tile_h, H), tx * P.tile_w:min((tx + 1) * P.tile_w, W)]
        ys, xs = ys.ravel(), xs.ravel()
        T = np.ones(len(xs))
        done = np.zeros(len(xs), bool)
        nc = np.zeros(len(xs), np.int64)
        bits = [0] * len(xs)
        for j, g in enumerate(lst[ts[t]:ts[t + 1]]):
            dx, dy = xs + 0.5 - pr["uv"][g, 0], ys + 0.5 - pr["uv"][g, 1]
            A, B, C = pr["conic"][g]
            p = -0.5 * (A * dx * dx + C * dy * dy) - B * dx * dy
            al = np.minimum(amax, pr["opacity"][g] * np.exp(p))
            ok = ~done & (p <= 0) & (al >= amin)
            tT = T * (1 - al)
            stop = ok & (tT < tmin)
            c = ok & ~stop
            done |= stop
            T = np.where(c, tT, T)
            nc = np.where(c, j + 1, nc)
            for q in np.nonzero(c)[0]:
                bits[q] |= 1 << j
        for q in range(len(xs)):
            comp[ys[q], xs[q]] = bits[q]
            ncon[ys[q], xs[q]] = nc[q]
    return comp, ncon


def test_gcount_by_hand(oracle_mod):
    """A 4 x 1 image.  Gaussian 0 (unit conic, opacity 0.5) is centred so that
    pixel 0 sees alpha = alpha_min (1 + 1e-7): pixel 0 is flagged, pixels 1-3
    are far from every threshold.  Gaussian 1 lies far away (alpha < 1e-30 at
    pixel 0), Gaussian 2 composites alpha 0.3 at every pixel.  The flagged
    pixel takes part in Gaussians 0 and 2: gcount = (1, 0, 1)."""
    O = oracle_mod
    P = O.Params()
    amin = float(F(P.alpha_min))
    d0 = math.sqrt(-2.0 * math.log(amin * (1 + 1e-7) / 0.5))
    cam = synth.plain_camera(4, 1, 10.0)
    proj = dict(status=np.zeros(3, np.int8), uv=np.array([[0.5 + d0, 0.5], [1e3, 0.5], [2.0, 0.5]]),
                conic=np.array([[1.0, 0.0, 1.0], [1.0, 0.0, 1.0], [1e-12, 0.0, 1e-12]]),
                opacity=np.array([0.5, 0.5, 0.3]), rgb=np.full((3, 3), 0.5))
    # one tile, depth order 0, 1, 2
    bins = (np.array([0, 3], np.int64), np.array([0, 1, 2], np.int32))
    out = O.render(proj, bins, cam, P)
    assert out["flags"][0, 0] != 0 and np.all(out["flags"][0, 1:] == 0)
    assert list(out["gcount"]) == [1, 0, 1]
    # the composited counts a by hand: G0 at pixels 0-3 (pixel 0 just above alpha_min), G2 everywhere
    assert list(out["a"]) == [4.0, 0.0, 4.0]


# ---- projection -------------------------------------------------------------------

def _fp32_radius(g, cam, P, tree):
    """ceil(3 sqrt(lambda_max)) in float32 from the float camera-space mean
    (nearest float to the exact one), by forming Sigma' as V V^T with
    V = J W R diag(s) and det by Cauchy-Binet ("V"), or as J W Sigma W^T J^T
    with Sigma formed first and det = a c - b^2 ("S")."""
    R64 = np.asarray(cam.R, np.float64).reshape(3, 3)
    t64 = np.asarray(g.mean, np.float64) @ R64.T + np.asarray(cam.t, np.float64)
    t = t64.astype(F)
    q = g.quat.astype(F)
    qn = np.sqrt(F(F(F(q[:, 0] * q[:, 0]) + F(q[:, 1] * q[:, 1])) + F(F(q[:, 2] * q[:, 2]) + F(q[:, 3] * q[:, 3]))))
    w, x, y, z = (F(q[:, i] / qn) for i in range(4))
    two = F(2)
    Q = [[F(1) - two * (y * y + z * z), two * (x * y - w * z), two * (x * z + w * y)],
         [two * (x * y + w * z), F(1) - two * (x * x + z * z), two * (y * z - w * x)],
         [two * (x * z - w * y), two * (y * z + w * x), F(1) - two * (x * x + y * y)]]
    s = np.exp(g.log_scale.astype(F)).astype(F)
    M = [[F(Q[i][j] * s[:, j]) for j in range(3)] for i in range(3)]
    fx, fy = F(cam.fx), F(cam.fy)
    limx = F(F(P.fov_clamp) * F(F(cam.width) / F(two * fx)))
    limy = F(F(P.fov_clamp) * F(F(cam.height) / F(two * fy)))
    xc = np.clip(F(t[:, 0] / t[:, 2]), -limx, limx).astype(F)
    yc = np.clip(F(t[:, 1] / t[:, 2]), -limy, limy).astype(F)
    tz2 = F(t[:, 2] * t[:, 2])
    j00, j02 = F(fx / t[:, 2]), F(-F(fx * F(xc * t[:, 2])) / tz2)
    j11, j12 = F(fy / t[:, 2]), F(-F(fy * F(yc * t[:, 2])) / tz2)
    W = np.asarray(cam.R, F).reshape(3, 3)
    T = [[F(F(j00 * W[0, k]) + F(j02 * W[2, k])) for k in range(3)],
         [F(F(j11 * W[1, k]) + F(j12 * W[2, k])) for k in range(3)]]
    dil = F(P.dilation)
    if tree == "V":
        V = [[F(F(F(T[r][0] * M[0][k]) + F(T[r][1] * M[1][k])) + F(T[r][2] * M[2][k])) for k in range(3)]
             for r in range(2)]
        s00 = F(F(F(V[0][0] * V[0][0]) + F(V[0][1] * V[0][1])) + F(V[0][2] * V[0][2]))
        s11 = F(F(F(V[1][0] * V[1][0]) + F(V[1][1] * V[1][1])) + F(V[1][2] * V[1][2]))
        a, c = F(s00 + dil), F(s11 + dil)
        m01 = F(F(V[0][0] * V[1][1]) - F(V[0][1] * V[1][0]))
        m02 = F(F(V[0][0] * V[1][2]) - F(V[0][2] * V[1][0]))
        m12 = F(F(V[0][1] * V[1][2]) - F(V[0][2] * V[1][1]))
        det = F(F(F(F(m01 * m01) + F(m02 * m02)) + F(m12 * m12)) + F(F(dil * F(s00 + s11)) + F(dil * dil)))
    else:
        Sg = [[F(F(F(M[i][0] * M[j][0]) + F(M[i][1] * M[j][1])) + F(M[i][2] * M[j][2])) for j in range(3)]
              for i in range(3)]

        def quad(r, cc):
            acc = F(0)
            for i in range(3):
                for j in range(3):
                    acc = F(acc + F(F(T[r][i] * Sg[i][j]) * T[cc][j]))
            return acc
        a, b, c = F(quad(0, 0) + dil), quad(0, 1), F(quad(1, 1) + dil)
        det = F(F(a * c) - F(b * b))
    mid = F(F(0.5) * F(a + c))
    disc = np.maximum(F(F(mid * mid) - det), F(0.1)).astype(F)
    lam = F(mid + np.sqrt(disc).astype(F))
    ext = F(F(3) * np.sqrt(lam).astype(F))
    return ext, t64


@pytest.mark.parametrize("scene", ["plain", "city"])
def test_radius_bound_covers_fp32_evaluations(oracle_mod, scene):
    O = oracle_mod
    if scene == "plain":
        g = synth.plain_scene(20000, seed=63)
        # a share of long thin needles
        g.log_scale[:3000, 0] = F(math.log(0.2))
        cam = synth.plain_camera(256, 256, 300.0)
        P = O.Params()
    else:
        g = synth.city_scene(200_000, seed=64)
        cam = synth.aerial_camera(seed=65)
        P = O.Params(lod_enable=True, lod_d0=1600.0, lod_Lmax=5)
    pr = O.project(O.gaussians64(g), cam, P)
    act = pr["status"] == O.ACTIVE
    assert act.sum() > 1000
    ext64, err = pr["extent"][:, 0], pr["extent"][:, 1]
    free = act & ((pr["tie"] & O.TIE_RADIUS) == 0)
    assert (act & ~free).sum() <= max(3, 5e-3 * act.sum())
    for tree in ("V", "S"):
        ext32, _ = _fp32_radius(g, cam, P, tree)
        d = np.abs(ext32.astype(np.float64) - ext64)
        # the running bound covers both evaluations at every active Gaussian
        assert np.all(d[act] <= err[act]), (tree, np.max(d[act] / err[act]))
        assert np.array_equal(np.ceil(ext32[free]).astype(np.int64), pr["radius"][free].astype(np.int64)), tree


def test_radius_flag_at_an_integer_extent(oracle_mod):
    """An isotropic Gaussian on the optical axis: Sigma' = (f s / z)^2 + 0.3 with
    the discriminant clamped, ext = 3 sqrt((f s / z)^2 + 0.3 + sqrt(0.1)).  The
    scale for ext = 12 exactly is flagged; one for ext = 12.01 is not."""
    O = oracle_mod
    cam = synth.plain_camera(64, 64, 300.0)
    P = O.Params()
    f, z, dil = float(F(300.0)), 3.0, float(F(0.3))

    def gauss(ext):
        s = math.sqrt((ext / 3.0) ** 2 - dil - math.sqrt(0.1)) * z / f
        g = synth.GaussianSet(mean=np.array([[0.0, 0.0, z]], F), log_scale=np.full((1, 3), math.log(s), F),
                              quat=np.array([[1, 0, 0, 0]], F), opacity_logit=np.zeros(1, F),
                              sh=np.zeros((1, 16, 3), F), lod=np.zeros(1, np.uint8))
        return O.project(O.gaussians64(g), cam, P)

    hit = gauss(12.0)
    assert abs(hit["extent"][0, 0] - 12.0) < 1e-5
    assert hit["tie"][0] & O.TIE_RADIUS
    miss = gauss(12.01)
    assert not miss["tie"][0] & O.TIE_RADIUS and miss["radius"][0] == 13


def test_lod_flag_at_a_half_integer_level(oracle_mod):
    """d0 / d = 2^(k + 1/2) puts log_2(d0 / d) on a rounding boundary: flagged;
    a distance 1e-4 relative away is not."""
    O = oracle_mod
    cam = synth.plain_camera(64, 64, 300.0)
    P = O.Params(lod_enable=True, lod_d0=16.0, lod_f=2.0, lod_Lmax=4)
    for d, flagged in ((16.0 / 2 ** 2.5, True), (16.0 / 2 ** 2.5 * (1 + 1e-4), False)):
        dz = float(F(d))
        g = synth.GaussianSet(mean=np.array([[0.0, 0.0, dz]], F), log_scale=np.full((1, 3), -4.0, F),
                              quat=np.array([[1, 0, 0, 0]], F), opacity_logit=np.zeros(1, F),
                              sh=np.zeros((1, 16, 3), F), lod=np.array([3], np.uint8))
        pr = O.project(O.gaussians64(g), cam, P)
        assert bool(pr["tie"][0] & O.TIE_LOD) == flagged, d


# ---- gradient conditioning bounds ---------------------------------------------------

def test_gradient_bounds_closed_form_isotropic(oracle_mod):
    """An isotropic Gaussian on the optical axis (identity rotation): V has the
    columns (f s / z) e_x, (f s / z) e_y and 0, so w_0, w_1 lie along the axes,
    w_2 = 0, and with dL/dC = 1 at every pixel every pixel term of dL/dA has
    one sign.  Then the log-scale bound is exactly (eps_sum + 2 prec_conic)
    |dL/dlog s_k| for the two visible axes, 0 for the axis along the view
    direction, and every rotation bound is 0 (no rotation moves the footprint)."""
    O = oracle_mod
    cam = synth.plain_camera(48, 48, 120.0)
    P = O.Params()
    g = synth.GaussianSet(mean=np.array([[0.0, 0.0, 3.0]], F), log_scale=np.full((1, 3), math.log(0.05), F),
                          quat=np.array([[1, 0, 0, 0]], F), opacity_logit=np.array([0.4], F),
                          sh=np.zeros((1, 16, 3), F), lod=np.zeros(1, np.uint8))
    g.sh[0, 0, :] = F(0.7)
    g64 = O.gaussians64(g)
    fwd = O.forward_view(g64, cam, P)
    grads = O.backward_view(g64, fwd, cam, P, np.ones((3, cam.height, cam.width)))
    og = O.grads_per_gaussian(grads)
    f = O.EPS_CONIC_SUM + 2 * P.prec_conic
    gls, bls = og["log_scale"][0], og["bounds"]["log_scale"][0]
    assert abs(gls[0]) > 0 and abs(gls[1]) > 0 and abs(gls[2]) < 1e-12 * abs(gls[0])
    np.testing.assert_allclose(bls[:2], f * np.abs(gls[:2]), rtol=1e-9)
    assert bls[2] == 0.0
    assert np.all(og["bounds"]["quat"][0] == 0.0)


def test_gradient_bounds_grow_with_cancellation(oracle_mod):
    """A long thin needle: its short axes' log-scale gradients are sums of
    pixel terms that nearly cancel, so their bounds exceed a small fraction of
    the gradient by the cancellation ratio, while the long axis stays bounded
    near (eps_sum + 2 prec_conic) |gradient|."""
    O = oracle_mod
    cam = synth.plain_camera(96, 96, 200.0)
    P = O.Params()
    rng = np.random.default_rng(66)
    half = math.radians(20.0)
    g = synth.GaussianSet(mean=np.array([[0.02, -0.01, 3.0]], F),
                          log_scale=np.array([[math.log(0.4), math.log(0.004), math.log(0.006)]], F),
                          quat=np.array([[math.cos(half), 0.1, 0.2, math.sin(half)]], F),
                          opacity_logit=np.array([0.4], F), sh=np.zeros((1, 16, 3), F), lod=np.zeros(1, np.uint8))
    g.sh[0, 0, :] = F(0.7)
    g64 = O.gaussians64(g)
    fwd = O.forward_view(g64, cam, P)
    grads = O.backward_view(g64, fwd, cam, P, rng.standard_normal((3, cam.height, cam.width)))
    og = O.grads_per_gaussian(grads)
    f = O.EPS_CONIC_SUM + 2 * P.prec_conic
    gls, bls = np.abs(og["log_scale"][0]), og["bounds"]["log_scale"][0]
    assert bls[0] < 50 * f * gls[0]
    assert max(bls[1] / gls[1], bls[2] / gls[2]) > 100 * f
