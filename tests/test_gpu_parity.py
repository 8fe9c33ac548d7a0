"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Bars: bit-exact for integer work (active records, tile rectangles and counts,
depth keys, sorted per-tile lists, n_contrib); images within 1e-4 max-abs;
gradients and importance scores within 1e-3 relative.  The oracle takes every
decision in FP64 and flags those within an FP32 renderer's error bound of
their boundary: a flagged projection decision must be one of the outcomes the
flag allows and is then taken into the oracle's projection; a flagged
compositing decision excludes its pixel.  Both stay rare.
"""
import dataclasses
import math

import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_13794_gb300 import binding as B
from paper_2605_13794_gb300 import synth
from tests.gpu_helpers import (ViewRun, assert_grad_close, assert_gaussian_grads_close, assert_param_grad_close, assert_record_precision,
                               capacity_for, footprint_power_err, gpu_params, grads_to_host, oracle_view_matched,
                               unpack_rect)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_13794_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()


def _compare_view(run: ViewRun, c, g64, cam, P, cull=None, check_image=True):
    """Compares one camera of a GPU run with the oracle; returns the oracle forward.

    Projection decisions (active set, rectangles, tile counts, depth keys) are
    exact outside the oracle's tie flags; a flagged decision must be one the
    flag allows and is then taken into the oracle's projection, so binning,
    image and everything downstream compare exactly or within tolerance."""
    fwd = oracle_view_matched(O, run, c, g64, cam, P, cull)
    pr = fwd["proj"]
    recs = run.records_of(c)
    both = np.nonzero(pr["status"] == O.ACTIVE)[0]
    assert sorted(recs.keys()) == both.tolist()
    ridx = np.array([recs[i] for i in both], np.int64)
    assert np.array_equal(run.tt[ridx].astype(np.int64), pr["tiles"][both].astype(np.int64))
    # continuous projected values: the mean is held to about 48 bits (u + u_lo);
    # the conic as A (dx + k dy)^2 + D dy^2 within the precision the compositing
    # flags allow for, and through the exponent it gives on each footprint's
    # 1- and 3-sigma ellipses
    assert_record_precision(run, ridx, pr, both, P)
    perr = footprint_power_err(run.rd0[ridx], run.rd1[ridx], run.rd2[ridx], pr["conic"][both], pr["uv"][both])
    assert perr.max(initial=0.0) <= 2e-4, perr.max()
    np.testing.assert_allclose(run.rd1[ridx, 1], pr["opacity"][both], rtol=1e-6, atol=1e-7)
    rgb = np.concatenate([run.rd1[ridx, 2:4], run.rd2[ridx, :1]], 1)
    np.testing.assert_allclose(rgb, pr["rgb"][both], rtol=0, atol=2e-5)
    # sorted per-tile lists: bit-exact, against the oracle's binning of its own
    # decisions and against its binning of the GPU's own FP32 records
    # (rectangle and depth key as the GPU computed them)
    ts, lst = fwd["bins"]
    glists = run.tile_lists(c)
    for t, gl in enumerate(glists):
        assert np.array_equal(gl, lst[ts[t]:ts[t + 1]].astype(np.int64)), f"tile {t} list differs"
    n = pr["status"].shape[0]
    own = dict(status=np.full(n, O.EMPTY, np.int8), rect=np.zeros((n, 4), np.int32),
               depth32=np.zeros(n, np.float32), tiles=np.zeros(n, np.int32))
    own["status"][both] = O.ACTIVE
    own["rect"][both] = unpack_rect(run.rect[ridx])
    own["depth32"][both] = run.depth_bits[ridx].view(np.float32)
    own["tiles"][both] = run.tt[ridx]
    ts2, lst2 = O.bin_tiles(own, cam, P)
    for t, gl in enumerate(glists):
        assert np.array_equal(gl, lst2[ts2[t]:ts2[t + 1]].astype(np.int64)), f"tile {t}: GPU binning of its own records"
    if not check_image:
        return fwd
    # image: 1e-4 max-abs outside flagged pixels
    ok = fwd["flags"] == 0
    assert ok.mean() > 0.99
    img = run.image(c)
    err = np.abs(img - fwd["image"]).max(axis=0)
    assert err[ok].max() <= 1e-4, f"image max err {err[ok].max():.3e}"
    assert np.abs(run.T_final(c) - fwd["T"])[ok].max() <= 1e-4
    assert np.array_equal(run.n_contrib_img(c)[ok], fwd["n_contrib"][ok].astype(np.int64))
    return fwd


def test_plain_view_forward_parity():
    g = synth.plain_scene()
    cam = synth.plain_camera()
    P = O.Params()
    run = ViewRun(g, [cam], P)
    assert run.counts["n_records"] == run.counts["records_needed"]
    _compare_view(run, 0, O.gaussians64(g), cam, P)


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.2, 0.5, 1.0)])
def test_ragged_image_and_background(bg):
    # 250 x 170: partial tiles on the right and bottom edges
    g = synth.plain_scene(6000, seed=7)
    cam = synth.plain_camera(250, 170, 260.0)
    P = O.Params(bg=bg)
    run = ViewRun(g, [cam], P)
    _compare_view(run, 0, O.gaussians64(g), cam, P)


def test_multi_camera_forward_parity():
    g = synth.plain_scene(8000, seed=9)
    cams = [synth.plain_camera(256, 256, 300.0), synth.plain_camera(200, 120, 180.0),
            synth.look_at_camera((0.6, -0.4, -0.5), (0.0, 0.0, 4.0), (0.0, -1.0, 0.0), 160, 144, 60.0)]
    P = O.Params()
    run = ViewRun(g, cams, P)
    g64 = O.gaussians64(g)
    for c, cam in enumerate(cams):
        _compare_view(run, c, g64, cam, P)


def test_lod_gate_and_cull_mask_parity():
    rng = np.random.default_rng(12)
    g = synth.plain_scene(8000, seed=13)
    g.lod[:] = rng.integers(0, 6, g.n).astype(np.uint8)
    cam = synth.plain_camera(192, 192, 220.0)
    cull = synth.random_cull_bits(g.n, 0.3, seed=14)
    # d0 so that distances 2..6 fall across levels 1..3
    P = O.Params(lod_enable=True, lod_d0=16.0, lod_Lmax=4, cull_enable=True)
    run = ViewRun(g, [cam], P, cull=cull)
    fwd = _compare_view(run, 0, O.gaussians64(g), cam, P, cull=cull)
    st = fwd["proj"]["status"]
    assert (st == O.GATED_LOD).sum() > 1000 and (st == O.GATED_CULL).sum() > 1000


@pytest.mark.parametrize("ncam", [1, 2])
def test_gate_bulk_copies_equal_plain_loads(ncam):
    """The view gate streams whole chunks of means and levels by bulk copies
    when the arrays are 16-byte aligned and by plain loads otherwise: both give
    the same candidates, records and image, bit for bit (a level array at an
    odd address takes the plain loads).  9000 Gaussians: eight whole chunks of
    1024 and a partial one."""
    rng = np.random.default_rng(41)
    g = synth.plain_scene(9000, seed=42)
    g.lod[:] = rng.integers(0, 6, g.n).astype(np.uint8)
    cams = [synth.plain_camera(160, 144, 200.0), synth.plain_camera(128, 96, 150.0)][:ncam]
    P = gpu_params(O.Params(lod_enable=True, lod_d0=16.0, lod_Lmax=4))
    gt = B.GaussianTensors.from_host(g)
    buf = torch.zeros(g.n + 16, dtype=torch.uint8, device="cuda")
    odd = buf[1:1 + g.n]
    odd.copy_(gt.lod)
    assert odd.data_ptr() % 16 != 0 and gt.lod.data_ptr() % 16 == 0
    npix = sum(c.width * c.height for c in cams)

    def run(gtx):
        ws = B.Workspace(**capacity_for(g.n, cams))
        ws.preprocess(gtx, cams, P, None)
        ws.bin_sort()
        rgb = torch.empty(3 * npix, device="cuda")
        ws.render_fwd(rgb)
        ws.sync_status()
        return rgb.cpu().numpy(), ws.counts()

    a, ca = run(gt)
    b, cb = run(dataclasses.replace(gt, lod=odd))
    for k in ("n_candidates", "n_records", "n_instances", "n_visible"):
        assert ca[k] == cb[k], k
    assert 0 < ca["n_records"] < g.n * ncam
    assert np.array_equal(a, b)


def test_long_tile_lists_sorted_by_depth():
    """Tiles whose lists exceed what one warp sorts in shared memory (512
    entries) are sorted in chunks merged through a scratch copy: every list
    equals the oracle's binning of the GPU's own records (rectangle and depth
    key as the GPU computed them), bit for bit, equal depths included."""
    g = synth.plain_scene(3000, seed=71)
    g.mean[:, :2] *= 0.05                       # every mean in front of a 48 x 48 view
    g.mean[1::2, 2] = g.mean[0::2, 2][: g.n // 2]  # pairs of equal depths
    g.log_scale[:] = np.float32(np.log(0.1))    # footprints over all nine tiles
    cam = synth.plain_camera(48, 48, 300.0)
    P = O.Params()
    run = ViewRun(g, [cam], P)
    recs = run.records_of(0)
    both = np.array(sorted(recs.keys()), np.int64)
    ridx = np.array([recs[i] for i in both], np.int64)
    n = g.n
    own = dict(status=np.full(n, O.EMPTY, np.int8), rect=np.zeros((n, 4), np.int32),
               depth32=np.zeros(n, np.float32), tiles=np.zeros(n, np.int32))
    own["status"][both] = O.ACTIVE
    own["rect"][both] = unpack_rect(run.rect[ridx])
    own["depth32"][both] = run.depth_bits[ridx].view(np.float32)
    own["tiles"][both] = run.tt[ridx]
    ts, lst = O.bin_tiles(own, cam, P)
    glists = run.tile_lists(0)
    assert max(len(l) for l in glists) > 2048  # three levels of merges
    for t, gl in enumerate(glists):
        assert np.array_equal(gl, lst[ts[t]:ts[t + 1]].astype(np.int64)), f"tile {t} list differs"


def test_cull_mark_equals_drop_for_training_and_off_for_importance():
    """GS_CULL_MARK keeps culled Gaussians in the lists, marked: the training
    render and its gradients are those of GS_CULL_DROP bit for bit, and the
    importance sweep on the same binning is that of GS_CULL_OFF bit for bit."""
    g = synth.plain_scene(4000, seed=31)
    cams = [synth.plain_camera(128, 112, 160.0), synth.plain_camera(96, 80, 120.0)]
    n, words = g.n, (g.n + 31) // 32
    rng = np.random.default_rng(32)
    cull = (rng.integers(0, 1 << 32, size=(2, words), dtype=np.uint64) &
            rng.integers(0, 1 << 32, size=(2, words), dtype=np.uint64)).astype(np.uint32) # ~25 % culled
    cull_t = torch.from_numpy(cull.view(np.int32).ravel()).cuda()
    P = O.Params(bg=(0.1, 0.2, 0.3))
    gt = B.GaussianTensors.from_host(g)
    npix = sum(c.width * c.height for c in cams)
    dL = torch.from_numpy(rng.standard_normal(3 * npix).astype(np.float32)).cuda()

    def run(mode):
        ws = B.Workspace(**capacity_for(n, cams))
        ws.preprocess(gt, cams, gpu_params(P, cull_enable=mode), cull_t if mode else None)
        ws.bin_sort()
        rgb, T = torch.empty(3 * npix, device="cuda"), torch.empty(npix, device="cuda")
        ws.render_fwd(rgb, T)
        out = dict(rgb=rgb.cpu().numpy(), T=T.cpu().numpy(), counts=ws.counts())
        grads, absg, reg = gt.zeros_like(), torch.zeros(n, device="cuda"), torch.zeros(1, device="cuda")
        ws.render_bwd(gt, dL, grads, accumulate=False, absgrad=absg, scale_reg_beta=10.0, scale_reg_value=reg)
        views = torch.zeros(n, device="cuda", dtype=torch.int32)
        ws.count_views(views)
        out.update(grads=grads_to_host(grads), absg=absg.cpu().numpy(), reg=reg.item(), views=views.cpu().numpy())
        out["imp"] = _importance(ViewRunLike(ws), n, len(cams))
        return out

    drop, mark, off = run(B.GS_CULL_DROP), run(B.GS_CULL_MARK), run(B.GS_CULL_OFF)
    assert mark["counts"]["n_records"] == off["counts"]["n_records"] > drop["counts"]["n_records"]
    assert mark["counts"]["n_visible"] == drop["counts"]["n_visible"]
    for k in ("rgb", "T", "absg", "views"):
        assert np.array_equal(mark[k], drop[k]), k
    assert mark["reg"] == drop["reg"]
    for k in mark["grads"]:
        assert np.array_equal(mark["grads"][k], drop["grads"][k]), k
    for k in off["imp"]:
        assert np.array_equal(mark["imp"][k], off["imp"][k]), k
    # and the marked render is the oracle's culled render
    g64 = O.gaussians64(g)
    Pc = O.Params(bg=(0.1, 0.2, 0.3), cull_enable=True)
    base = 0
    for c, cam in enumerate(cams):
        fwd = O.forward_view(g64, cam, Pc, cull[c])
        hw = cam.width * cam.height
        img = mark["rgb"][3 * base:3 * (base + hw)].reshape(3, cam.height, cam.width)
        ok = fwd["flags"] == 0
        assert ok.mean() > 0.99
        assert np.abs(img - fwd["image"]).max(axis=0)[ok].max() <= 1e-4
        base += hw


@pytest.mark.parametrize("mode", [B.GS_CULL_MARK, B.GS_CULL_OFF])
def test_fused_forward_importance_matches_separate(mode):
    """gs_render_fwd_importance: the image, T_final and n_contrib of gs_render_fwd
    and the importance outputs of gs_importance's own raster, bit for bit, on a
    two-camera scene with a Cull column; the backward after it is unchanged."""
    g = synth.plain_scene(4000, seed=33)
    cams = [synth.plain_camera(128, 112, 160.0), synth.plain_camera(96, 80, 120.0)]
    n, words = g.n, (g.n + 31) // 32
    rng = np.random.default_rng(34)
    cull = (rng.integers(0, 1 << 32, size=(2, words), dtype=np.uint64) &
            rng.integers(0, 1 << 32, size=(2, words), dtype=np.uint64)).astype(np.uint32)
    cull_t = torch.from_numpy(cull.view(np.int32).ravel()).cuda()
    P = O.Params(bg=(0.1, 0.2, 0.3))
    gt = B.GaussianTensors.from_host(g)
    npix = sum(c.width * c.height for c in cams)
    dL = torch.from_numpy(rng.standard_normal(3 * npix).astype(np.float32)).cuda()

    def run(fused):
        ws = B.Workspace(**capacity_for(n, cams))
        ws.preprocess(gt, cams, gpu_params(P, cull_enable=mode), cull_t if mode else None)
        ws.bin_sort()
        rgb, T = torch.empty(3 * npix, device="cuda"), torch.empty(npix, device="cuda")
        (ws.render_fwd_importance if fused else ws.render_fwd)(rgb, T)
        nc = ws.read_buffer(B.GS_BUF_N_CONTRIB, np.uint32, npix)
        grads = gt.zeros_like()
        ws.render_bwd(gt, dL, grads, accumulate=False)
        imp = _importance(ViewRunLike(ws), n, len(cams))
        return rgb.cpu().numpy(), T.cpu().numpy(), nc, grads_to_host(grads), imp

    sep, fus = run(False), run(True)
    for k in range(3):
        assert np.array_equal(sep[k], fus[k])
    for k in sep[3]:
        assert np.array_equal(sep[3][k], fus[3][k]), k
    for k in sep[4]:
        assert np.array_equal(sep[4][k], fus[4][k]), k


def test_importance_on_a_second_stream_matches_one_stream():
    """gs_importance shares no scratch with the training pass: forked onto a
    second stream after gs_bin_sort, beside gs_render_fwd, gs_photometric_loss,
    gs_render_bwd_compact and gs_adam_step_compact of the same binning, and
    captured with them as one graph (torch's, and the library's with per-kernel
    priorities), three steps (each gated by the previous step's Cull column)
    give the one-stream results bit for bit."""
    g = synth.plain_scene(20000, seed=35)
    cams = [synth.plain_camera(320, 240, 300.0)]
    cam = cams[0]
    n, words, npix = g.n, (g.n + 31) // 32, cam.width * cam.height
    rng = np.random.default_rng(36)
    target = torch.from_numpy(rng.random((1, 3, cam.height, cam.width), dtype=np.float32)).cuda()
    P = O.Params(bg=(0.1, 0.2, 0.3))
    lr = [1e-3, 5e-3, 1e-3, 5e-2, 2.5e-3]

    def run(mode):
        gt = B.GaussianTensors.from_host(g)
        m, v = gt.zeros_like(), gt.zeros_like()
        ws = B.Workspace(**capacity_for(n, cams))
        side = torch.cuda.Stream() if mode != "one" else None
        rgb, T, dL = (torch.empty(3 * npix, device="cuda"), torch.empty(npix, device="cuda"),
                      torch.empty(3 * npix, device="cuda"))
        loss, reg = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
        s = torch.zeros(n, device="cuda")
        crad, cvis = (torch.zeros(n, device="cuda", dtype=torch.int32) for _ in range(2))
        cull = torch.zeros(words, device="cuda", dtype=torch.int32)
        ws.preprocess(gt, cams, gpu_params(P), None)
        ws.bin_sort()
        ws.importance(cull_out=cull)
        ws.upload_cameras(cams, gpu_params(P, cull_enable=B.GS_CULL_MARK))
        losses = []

        def body():
            main = torch.cuda.current_stream() # the capture stream inside the graph capture
            ws.preprocess_uploaded(gt, gpu_params(P, cull_enable=B.GS_CULL_MARK), cull)
            ws.bin_sort()
            if side is not None:
                side.wait_stream(main)
                ws.importance(s_accum=s, crad=crad, cvis=cvis, cull_out=cull, stream=side)
            ws.render_fwd(rgb, T)
            ws.photometric_loss(rgb.view(1, 3, cam.height, cam.width), target, 0.2, loss, dL)
            ws.render_bwd_compact(gt, dL, scale_reg_beta=10.0, scale_reg_value=reg)
            ws.adam_step_compact(gt, m, v, lr, 0)
            if side is None:
                ws.importance(s_accum=s, crad=crad, cvis=cvis, cull_out=cull)
            else:
                main.wait_stream(side)

        if mode == "graph":
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph):
                body()
            torch.cuda.synchronize()
        elif mode == "gs_graph": # the library's graph, the step on a high-priority stream
            torch.cuda.synchronize()
            graph = B.Graph()
            with graph.capture(torch.cuda.Stream(priority=-1)):
                body()
            torch.cuda.synchronize()
        for _ in range(3):
            if mode == "graph":
                graph.replay()
            elif mode == "gs_graph":
                graph.launch()
            else:
                body()
            losses.append(loss.clone())
        torch.cuda.synchronize()
        ws.sync_status()
        if mode == "gs_graph":
            graph.close()
        out = {f"p_{k}": t.cpu().numpy() for k, t in zip(("mean", "log_scale", "quat", "opacity_logit", "sh"),
                                                          gt.params())}
        out.update({f"m_{k}": t for k, t in grads_to_host(m).items()})
        out.update(rgb=rgb.cpu().numpy(), loss=torch.cat(losses).cpu().numpy(), reg=reg.cpu().numpy(),
                   s=s.cpu().numpy(), crad=crad.cpu().numpy(), cvis=cvis.cpu().numpy(), cull=cull.cpu().numpy())
        ws.close()
        return out

    one = run("one")
    assert one["crad"].sum() > 0 and one["cvis"].sum() > 0
    for mode in ("two", "graph", "gs_graph"):
        other = run(mode)
        for k in one:
            assert np.array_equal(one[k], other[k]), (mode, k)


class ViewRunLike:
    """The one attribute _importance needs from a ViewRun."""

    def __init__(self, ws):
        self.ws = ws


def test_empty_and_fully_gated_scenes():
    cam = synth.plain_camera(64, 48, 100.0)
    P = O.Params()
    g = synth.plain_scene(500, seed=15)
    g.mean[:, 2] = -1.0  # all behind the camera
    run = ViewRun(g, [cam], P)
    assert run.counts["n_records"] == 0 and run.counts["n_instances"] == 0
    assert np.allclose(run.image(0), 0.0) and np.allclose(run.T_final(0), 1.0)
    g0 = synth.plain_scene(0, seed=16)
    run0 = ViewRun(g0, [cam], P, cap=capacity_for(1, [cam]))
    assert run0.counts["n_records"] == 0 and np.allclose(run0.T_final(0), 1.0)


def test_capacity_overflow_is_reported():
    g = synth.plain_scene(4000, seed=17)
    cam = synth.plain_camera()
    P = O.Params()
    cap = capacity_for(g.n, [cam], instances=2000)
    with pytest.raises(B.GSError) as ei:
        ViewRun(g, [cam], P, cap=cap)
    assert ei.value.code == B.GS_ERR_CAPACITY


def _backward(run: ViewRun, dL):
    grads = run.gt.zeros_like()
    dLt = torch.from_numpy(np.ascontiguousarray(dL, np.float32).ravel()).cuda()
    run.ws.render_bwd(run.gt, dLt, grads, accumulate=False)
    run.ws.sync_status()
    return grads_to_host(grads)


@pytest.mark.parametrize("seed", [21, 22])
def test_backward_parity(seed):
    g = synth.plain_scene(3000, seed=seed)
    cam = synth.plain_camera(128, 112, 160.0)
    P = O.Params()
    run = ViewRun(g, [cam], P)
    g64 = O.gaussians64(g)
    fwd = _compare_view(run, 0, g64, cam, P)
    dL = np.random.default_rng(seed + 100).standard_normal((3, cam.height, cam.width))
    gg = _backward(run, dL)
    og = O.grads_per_gaussian(O.backward_view(g64, fwd, cam, P, dL))
    assert_gaussian_grads_close(gg, og)


def test_backward_parity_on_deep_lists():
    """Deep tile lists: 40k faint Gaussians (opacity about 0.05) packed into the
    middle of a 96x80 view, so each pixel's walk passes about two thousand
    entries (n_contrib) and composites many of them.  The adjoint's slots then
    sum moments over many composited pairs per entry and the reverse walk
    recovers T through long chains of divisions; the gradients stay within the
    parity rules."""
    g = synth.plain_scene(40000, seed=27)
    rng = np.random.default_rng(28)
    g.mean[:, :2] *= np.float32(0.5)
    g.opacity_logit[:] = (np.float32(-3.0) + np.float32(0.5) * rng.standard_normal(g.n)).astype(np.float32)
    cam = synth.plain_camera(96, 80, 160.0)
    P = O.Params()
    run = ViewRun(g, [cam], P)
    g64 = O.gaussians64(g)
    fwd = _compare_view(run, 0, g64, cam, P)
    assert run.n_contrib.mean() > 100  # deep lists indeed
    dL = rng.standard_normal((3, cam.height, cam.width))
    gg = _backward(run, dL)
    og = O.grads_per_gaussian(O.backward_view(g64, fwd, cam, P, dL))
    assert_gaussian_grads_close(gg, og)


def test_backward_fragment_counts_and_kernel_timing():
    """The backward's work counters: fragments is the sum of n_contrib (integer,
    exact); composited is the number of composited (pixel, Gaussian) pairs, the
    sum of the oracle's per-Gaussian pixel counts a (Sec. 3.2) up to the pairs of
    flagged pixels.  Timing brackets exactly the timed launches."""
    g = synth.plain_scene(3000, seed=25)
    cam = synth.plain_camera(144, 104, 160.0)
    P = O.Params()
    run = ViewRun(g, [cam], P)
    fwd = O.forward_view(O.gaussians64(g), cam, P)
    dL = np.random.default_rng(26).standard_normal((3, cam.height, cam.width))
    assert run.ws.kernel_time(B.GS_KT_RENDER_BWD) == (0.0, 0)
    run.ws.kernel_timing(True)
    _backward(run, dL)
    _backward(run, dL)
    ms, n = run.ws.kernel_time(B.GS_KT_RENDER_BWD)
    assert n == 2 and ms > 0.0
    assert run.ws.kernel_time(B.GS_KT_RENDER_FWD) == (0.0, 0)
    run.ws.kernel_timing(False)
    assert run.ws.kernel_time(B.GS_KT_RENDER_BWD) == (0.0, 0)
    c = run.ws.counts()
    # two backward launches since the preprocess
    assert c["fragments"] == 2 * int(run.n_contrib.astype(np.int64).sum())
    comp = c["composited"] // 2
    assert c["composited"] % 2 == 0
    # a selection of kernels: the backward is not timed when only the forward is
    run.ws.kernel_timing(True, kernels=[B.GS_KT_RENDER_FWD])
    _backward(run, dL)
    assert run.ws.kernel_time(B.GS_KT_RENDER_BWD) == (0.0, 0)
    run.ws.kernel_timing(True, kernels=[B.GS_KT_RENDER_BWD])
    _backward(run, dL)
    assert run.ws.kernel_time(B.GS_KT_RENDER_BWD)[1] == 1
    run.ws.kernel_timing(False)
    assert comp <= c["fragments"] // 2
    ref = int(round(fwd["a"].sum()))
    assert abs(comp - ref) <= int(fwd["gcount"].sum()) + 0, (comp, ref)
    assert comp > 0


def test_backward_multi_camera_accumulates():
    g = synth.plain_scene(3000, seed=23)
    cams = [synth.plain_camera(128, 128, 160.0), synth.plain_camera(96, 80, 120.0)]
    P = O.Params(bg=(0.1, 0.2, 0.3))
    run = ViewRun(g, cams, P)
    g64 = O.gaussians64(g)
    rng = np.random.default_rng(24)
    dLs = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    gg = _backward(run, np.concatenate([d.ravel() for d in dLs]))
    og = O.zero_grads(g.n)
    for c, cam in enumerate(cams):
        fwd = _compare_view(run, c, g64, cam, P)
        O.backward_view(g64, fwd, cam, P, dLs[c], og)
    og = O.grads_per_gaussian(og)
    assert_gaussian_grads_close(gg, og)


def test_deterministic_reruns():
    g = synth.plain_scene(5000, seed=25)
    cam = synth.plain_camera()
    P = O.Params()
    dL = np.random.default_rng(26).standard_normal((3, cam.height, cam.width))
    outs = []
    for _ in range(2):
        run = ViewRun(g, [cam], P)
        gg = _backward(run, dL)
        outs.append((run.image(0), gg))
    assert np.array_equal(outs[0][0], outs[1][0])
    for k in outs[0][1]:
        assert np.array_equal(outs[0][1][k], outs[1][1][k]), k


def _importance(run: ViewRun, n, ncam):
    dev = "cuda"
    w = torch.zeros(ncam * n, device=dev)
    a = torch.zeros(ncam * n, device=dev, dtype=torch.int32)
    s = torch.zeros(n, device=dev)
    crad = torch.zeros(n, device=dev, dtype=torch.int32)
    cvis = torch.zeros(n, device=dev, dtype=torch.int32)
    words = (n + 31) // 32
    cull = torch.zeros(ncam * words, device=dev, dtype=torch.int32)
    run.ws.importance(w, a, s, crad, cvis, cull)
    run.ws.sync_status()
    h = lambda t: t.cpu().numpy()
    return dict(w=h(w).reshape(ncam, n).astype(np.float64), a=h(a).reshape(ncam, n), s=h(s).astype(np.float64),
                crad=h(crad), cvis=h(cvis), cull=h(cull).view(np.uint32).reshape(ncam, words))


def _check_visible_set(vis_gpu, w_ref, vis_mass):
    """c^vis validity: the GPU set differs from the oracle's only by entries
    whose w is within 1e-3 of the oracle's cut value, and carries the mass."""
    vis_ref = O.visible_top_mass(w_ref, vis_mass)
    diff = np.nonzero(vis_gpu != vis_ref)[0]
    if vis_ref.any():
        cut = w_ref[vis_ref].min()
        assert np.all(np.abs(w_ref[diff] - cut) <= 1e-3 * cut + 1e-12), diff[:10]
    total = w_ref.sum()
    assert w_ref[vis_gpu].sum() >= vis_mass * total * (1 - 1e-5)
    assert not np.any(vis_gpu & (w_ref == 0))


def _check_cull_against_own_w(vis_gpu, w_gpu, vis_mass):
    """The Cull column is the 99 %-mass selection of the GPU's own w: the GPU's
    fixed-point prefix sums and the oracle's FP64 ones may put the cut one
    place apart, never more."""
    w64 = np.asarray(w_gpu, np.float64)
    mine = O.visible_top_mass(w64, vis_mass)
    pos = np.nonzero(w64 > 0)[0]
    order = pos[np.lexsort((pos, -w64[pos]))]
    k = int(mine.sum())
    diff = set(np.nonzero(vis_gpu != mine)[0].tolist())
    if len(order):
        assert diff <= {int(order[k - 1]), int(order[min(k, len(order) - 1)])} and len(diff) <= 1, sorted(diff)[:10]
    else:
        assert not diff


def test_importance_parity():
    """w and a per view, s, c^rad, c^vis and the Cull columns against the
    oracle.  A Gaussian on no flagged pixel (gcount 0) has w within the
    gradient rule and a exact; on a flagged pixel an undecided fragment may
    move a by one and w by one fragment's alpha T (< 1e-2), per such pixel."""
    g = synth.plain_scene(6000, seed=31)
    cams = [synth.plain_camera(), synth.plain_camera(160, 200, 200.0)]
    P = O.Params()
    run = ViewRun(g, cams, P)
    g64 = O.gaussians64(g)
    imp = _importance(run, g.n, len(cams))
    acc = O.new_importance(g.n)
    vm = float(np.float32(P.vis_mass))
    gcount = np.zeros(g.n, np.int64)
    bound = np.zeros(g.n)
    for c, cam in enumerate(cams):
        fwd = _compare_view(run, c, g64, cam, P, check_image=False)
        O.importance_update(acc, fwd["w"], fwd["a"], fwd["proj"], vm, float(np.float32(P.eps_score)))
        cnt = fwd["gcount"].astype(np.int64)
        gcount += cnt
        free = cnt == 0
        wg, ag, ao = imp["w"][c], imp["a"][c].astype(np.int64), fwd["a"].astype(np.int64)
        assert_grad_close(f"w[{c}]", np.where(free, wg, 0.0), np.where(free, fwd["w"], 0.0))
        assert np.array_equal(ag[free], ao[free])
        assert np.all(np.abs(ag - ao) <= cnt)
        assert np.all(np.abs(wg - fwd["w"]) <= 1e-3 * np.abs(fwd["w"]) + 1e-2 * cnt + 1e-9)
        # what the undecided fragments of this view can move s_i = sum w / (a + eps) by
        cf = cnt.astype(np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            hi = np.where(ao - cnt > 0, (fwd["w"] + 1e-2 * cf) / (ao - cnt), np.inf) - np.where(ao > 0, fwd["w"] / np.maximum(ao, 1), 0)
        bound += np.where(cnt > 0, hi, 0.0)
        vis_gpu = ~synth.unpack_bits(imp["cull"][c], g.n)
        _check_visible_set(vis_gpu, fwd["w"], vm)
        _check_cull_against_own_w(vis_gpu, wg, vm)
    free = gcount == 0
    assert free.sum() > 0.75 * (acc["crad"] > 0).sum()
    assert_grad_close("s", np.where(free, imp["s"], 0.0), np.where(free, acc["s"], 0.0))
    assert np.all(np.abs(imp["s"] - acc["s"]) <= 1e-3 * acc["s"] + bound + 1e-9)
    assert np.array_equal(imp["crad"], acc["crad"])
    assert np.abs(imp["cvis"] - acc["cvis"]).max() <= 1


def test_photometric_loss_parity():
    rng = np.random.default_rng(41)
    B_, H, W = 2, 70, 90
    x = rng.uniform(0, 1, (B_, 3, H, W)).astype(np.float32)
    y = rng.uniform(0, 1, (B_, 3, H, W)).astype(np.float32)
    ws = B.Workspace(**capacity_for(1, [synth.plain_camera(W, H)] * B_))
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    loss = torch.zeros(1, device="cuda")
    dL = torch.empty_like(xt)
    ws.photometric_loss(xt, yt, 0.2, loss, dL)
    torch.cuda.synchronize()
    L_ref, g_ref = O.photometric_loss(x, y, lam=float(np.float32(0.2)))
    assert abs(loss.item() - L_ref) <= 1e-5 * abs(L_ref)
    assert_grad_close("dL/dimage", dL.double().cpu().numpy(), g_ref, rtol=1e-3)


def test_adam_parity():
    rng = np.random.default_rng(42)
    sizes = [1000, 37, 4096]
    groups, host = [], []
    for k, n in enumerate(sizes):
        p, g = rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32)
        m, v = (0.1 * rng.standard_normal(n)).astype(np.float32), np.abs(0.1 * rng.standard_normal(n)).astype(np.float32)
        host.append((p, g, m, v, 1e-3 * (k + 1)))
        groups.append([torch.from_numpy(a).cuda() for a in (p, g, m, v)] + [1e-3 * (k + 1), 0.9, 0.999, 1e-15])
    B.adam_step(groups, step=3)
    torch.cuda.synchronize()
    for (p, g, m, v, lr), dev in zip(host, groups):
        pr, mr, vr = O.adam_step(p, g, m, v, 3, float(np.float32(lr)), float(np.float32(0.9)), float(np.float32(0.999)),
                                 float(np.float32(1e-15)))
        np.testing.assert_allclose(dev[0].cpu().numpy(), pr, rtol=1e-5, atol=1e-7)
        np.testing.assert_allclose(dev[2].cpu().numpy(), mr, rtol=1e-5, atol=1e-8)
        np.testing.assert_allclose(dev[3].cpu().numpy(), vr, rtol=1e-5, atol=1e-10)


def test_scale_regulariser_parity():
    g = synth.plain_scene(2000, seed=43)
    cam = synth.plain_camera()
    P = O.Params()
    run = ViewRun(g, [cam], P)
    grads = run.gt.zeros_like()
    val = torch.zeros(1, device="cuda")
    zero = torch.zeros(3 * cam.pixels, device="cuda")
    run.ws.render_bwd(run.gt, zero, grads, accumulate=False, scale_reg_beta=10.0, scale_reg_value=val)
    torch.cuda.synchronize()
    pr = O.project(O.gaussians64(g), cam, P)
    vis = pr["status"] == O.ACTIVE
    ref_val, ref_g = O.scale_regulariser(g.log_scale.T.astype(np.float64), vis, beta=10.0)
    assert abs(val.item() - ref_val) <= 1e-5 * ref_val
    assert_grad_close("log_scale", grads.log_scale.double().cpu().numpy(), ref_g.T)


def test_fused_backward_adam_matches_unfused():
    """gs_render_bwd_adam == gs_render_bwd followed by gs_adam_step, bit for bit
    (the same gradient arithmetic feeds the same update)."""
    g = synth.plain_scene(4000, seed=44)
    cam = synth.plain_camera(160, 144, 200.0)
    P = O.Params()
    run = ViewRun(g, [cam], P)
    rng = np.random.default_rng(45)
    dL = torch.from_numpy(rng.standard_normal(3 * cam.pixels).astype(np.float32)).cuda()
    lr = [1e-2, 5e-3, 1e-3, 5e-2, 2.5e-3]
    names = ("mean", "log_scale", "quat", "opacity_logit", "sh")

    def state():
        m = run.gt.zeros_like()
        v = run.gt.zeros_like()
        for t in m.params():
            t.copy_(torch.from_numpy((0.01 * rng.standard_normal(t.numel())).astype(np.float32)).view_as(t))
        for t in v.params():
            t.copy_(torch.from_numpy(np.abs(0.01 * rng.standard_normal(t.numel())).astype(np.float32)).view_as(t))
        return m, v

    m0, v0 = state()
    # unfused: dense gradients, then the dense Adam step
    pa = B.GaussianTensors(*[t.clone() for t in run.gt.params()], None)
    ma, va = B.GaussianTensors(*[t.clone() for t in m0.params()], None), B.GaussianTensors(*[t.clone() for t in v0.params()], None)
    grads = run.gt.zeros_like()
    run.ws.render_bwd(run.gt, dL, grads, accumulate=False)
    B.adam_step([(p, gr, m, v, lr[k], 0.9, 0.999, 1e-15) for k, (p, gr, m, v) in
                 enumerate(zip(pa.params(), grads.params(), ma.params(), va.params()))], step=3)
    # fused: compact rows consumed by the streaming update
    pb = B.GaussianTensors(*[t.clone() for t in run.gt.params()], None)
    mb, vb = B.GaussianTensors(*[t.clone() for t in m0.params()], None), B.GaussianTensors(*[t.clone() for t in v0.params()], None)
    run.ws.render_bwd_adam(pb, dL, mb, vb, lr, step=3)
    run.ws.sync_status()
    for k, name in enumerate(names):
        assert torch.equal(pa.params()[k], pb.params()[k]), name
        assert torch.equal(ma.params()[k], mb.params()[k]), name
        assert torch.equal(va.params()[k], vb.params()[k]), name
    # and the update agrees with the oracle's gradients and Adam
    g64 = O.gaussians64(g)
    fwd = O.forward_view(g64, cam, P)
    og = O.grads_per_gaussian(O.backward_view(g64, fwd, cam, P, dL.double().cpu().numpy().reshape(3, cam.height, cam.width)))
    for k, name in enumerate(names):
        p_ref, _, _ = O.adam_step(getattr(g, name), og[name], m0.params()[k].cpu().numpy(), v0.params()[k].cpu().numpy(),
                                  3, float(np.float32(lr[k])))
        step_ref = p_ref - getattr(g, name)
        step_gpu = pb.params()[k].double().cpu().numpy() - getattr(g, name)
        # the step is m/sqrt(v): elementwise it is ill-conditioned where 0.9 m0 and 0.1 g cancel,
        # so only the tensor-wide rule applies here (the gradients are compared elementwise above)
        assert_grad_close(f"adam step {name}", step_gpu, step_ref, rtol=1e-3, big=1.0)
