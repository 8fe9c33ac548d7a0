"""Batched rendering through the C ABI: tile shapes, several cameras of uneven
resolution in one pass, and the multi-view training step run eagerly and as
a replayed CUDA graph."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_13794_gb300 import binding as B
from paper_2605_13794_gb300 import synth
from paper_2605_13794_gb300.train import TrainStep
from tests.gpu_helpers import (ViewRun, assert_grad_close, assert_gaussian_grads_close, assert_param_grad_close, capacity_for, gpu_params,
                               grads_to_host)
from tests.test_gpu_parity import _compare_view

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_13794_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()

TILE_SHAPES = [(16, 16), (32, 8), (8, 32), (32, 16), (16, 8), (8, 16)]


def _uneven_cameras():
    return [synth.plain_camera(250, 170, 260.0), synth.plain_camera(96, 80, 120.0),
            synth.look_at_camera((0.6, -0.4, -0.5), (0.0, 0.0, 4.0), (0.0, -1.0, 0.0), 161, 143, 60.0)]


@pytest.mark.parametrize("tw,th", TILE_SHAPES)
def test_tile_shapes_forward_backward_importance(tw, th):
    g = synth.plain_scene(6000, seed=51)
    cams = _uneven_cameras()
    P = O.Params(tile_w=tw, tile_h=th)
    run = ViewRun(g, cams, P)
    g64 = O.gaussians64(g)
    fwds = [_compare_view(run, c, g64, cam, P) for c, cam in enumerate(cams)]
    # backward over all three views at once
    rng = np.random.default_rng(52)
    dLs = [rng.standard_normal((3, c.height, c.width)) for c in cams]
    grads = run.gt.zeros_like()
    dLt = torch.from_numpy(np.concatenate([d.ravel() for d in dLs]).astype(np.float32)).cuda()
    run.ws.render_bwd(run.gt, dLt, grads, accumulate=False)
    run.ws.sync_status()
    og = O.zero_grads(g.n)
    for c, cam in enumerate(cams):
        O.backward_view(g64, fwds[c], cam, P, dLs[c], og)
    og = O.grads_per_gaussian(og)
    gg = grads_to_host(grads)
    assert_gaussian_grads_close(gg, og)
    # importance per view
    w = torch.zeros(len(cams) * g.n, device="cuda")
    a = torch.zeros(len(cams) * g.n, device="cuda", dtype=torch.int32)
    run.ws.importance(w=w, a=a)
    run.ws.sync_status()
    wv, av = w.view(len(cams), g.n).double().cpu().numpy(), a.view(len(cams), g.n).cpu().numpy()
    for c in range(len(cams)):
        assert_grad_close(f"w[{c}]", wv[c], fwds[c]["w"])
        assert (av[c] != fwds[c]["a"]).sum() <= 1e-3 * max(1, (fwds[c]["a"] > 0).sum())


def test_tile_shapes_give_the_same_image_away_from_tile_dependent_fragments():
    # Low opacity keeps every alpha >= 1/255 fragment inside the 3-sigma box,
    # so every tiling composites the same fragments: images agree to rounding.
    g = synth.plain_scene(5000, seed=53)
    g.opacity_logit[:] = np.minimum(g.opacity_logit, np.float32(np.log(0.34 / 0.66)))
    cams = _uneven_cameras()
    imgs = []
    for tw, th in TILE_SHAPES:
        run = ViewRun(g, cams, O.Params(tile_w=tw, tile_h=th))
        imgs.append(torch.cat([run.rgb]).double().cpu().numpy())
    for im in imgs[1:]:
        assert np.abs(im - imgs[0]).max() <= 1e-5


def _views(k, n=2, W=112, H=96):
    rng = np.random.default_rng(1000 + k)
    cams = []
    for _ in range(n):
        eye = (rng.uniform(-0.6, 0.6), rng.uniform(-0.6, 0.6), rng.uniform(-1.0, -0.3))
        cams.append(synth.look_at_camera(eye, (0.0, 0.0, 4.0), (0.0, -1.0, 0.0), W, H, 60.0))
    return cams


def _targets(cams, seed):
    return torch.from_numpy(np.stack([synth.noise_target(c.width, c.height, seed=seed + i)
                                      for i, c in enumerate(cams)]).astype(np.float32)).cuda()


LR = [1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3]


def test_graph_replay_equals_eager():
    g = synth.plain_scene(4000, seed=54)
    params = B.RenderParams()
    ga, gb = B.GaussianTensors.from_host(g), B.GaussianTensors.from_host(g)
    cams0 = _views(0)
    eager = TrainStep(ga, cams0, _targets(cams0, 10), params, LR)
    graph = TrainStep(gb, cams0, _targets(cams0, 10), params, LR)
    eager.run(step=1)
    graph.run(step=1)           # first step eagerly: sets the device step counter
    graph.capture()
    for k in range(1, 5):
        cams = _views(k)
        tg = _targets(cams, 10 + 7 * k)
        eager.set_views(cams, tg)
        eager.run()             # step 0: continue the device counter, like the graph
        graph.set_views(cams, tg)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(eager.loss, graph.loss), k
    eager.ws.sync_status()
    graph.ws.sync_status()
    for a, b in zip(ga.params(), gb.params()):
        assert torch.equal(a, b)
    for a, b in zip(eager.m.params() + eager.v.params(), graph.m.params() + graph.v.params()):
        assert torch.equal(a, b)


def test_upload_is_refused_inside_capture():
    g = B.GaussianTensors.from_host(synth.plain_scene(500, seed=55))
    cams = _views(0)
    step = TrainStep(g, cams, _targets(cams, 3), B.RenderParams(), LR)
    s = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with pytest.raises(B.GSError):
        with torch.cuda.graph(graph, stream=s):
            step.ws.upload_cameras(cams, step.params)
    torch.cuda.synchronize()


def test_multi_view_train_step_against_oracle():
    """One step of L1 + 0.2 D-SSIM + scale regulariser over 3 views, then Adam
    from zero moments: loss and the updated parameters against the oracle."""
    g = synth.plain_scene(3000, seed=56)
    cams = _views(3, n=3)
    targets = _targets(cams, 20)
    params = B.RenderParams()
    gt = B.GaussianTensors.from_host(g)
    step = TrainStep(gt, cams, targets, params, LR)
    step.run(step=1)
    step.ws.sync_status()
    torch.cuda.synchronize()
    # oracle: per-view forward, the batch loss of Eq. 4, per-view adjoints, Eq. 5, Adam
    P = O.Params()
    g64 = O.gaussians64(g)
    fwds = [O.forward_view(g64, c, P) for c in cams]
    imgs = np.stack([f["image"] for f in fwds]).astype(np.float32)
    L_ref, dimg = O.photometric_loss(imgs, targets.cpu().numpy(), lam=float(np.float32(0.2)))
    assert abs(step.loss.item() - L_ref) <= 1e-4 * abs(L_ref)
    og = O.zero_grads(g.n)
    for c, cam in enumerate(cams):
        O.backward_view(g64, fwds[c], cam, P, dimg[c], og)
    vis = np.zeros(g.n, bool)
    for f in fwds:
        vis |= f["proj"]["status"] == O.ACTIVE
    reg, reg_g = O.scale_regulariser(g.log_scale.T.astype(np.float64), vis, beta=10.0)
    assert abs(step.reg.item() - reg) <= 1e-5 * reg
    og["log_scale"] += reg_g
    og = O.grads_per_gaussian(og)
    names = ("mean", "log_scale", "quat", "opacity_logit", "sh")
    for k, name in enumerate(names):
        p0 = getattr(g, name).astype(np.float64)
        p_ref, _, _ = O.adam_step(p0, og[name], np.zeros_like(p0), np.zeros_like(p0), 1, float(np.float32(LR[k])))
        got = gt.params()[k].double().cpu().numpy()
        # first step from zero moments: -lr g / (|g| + eps), i.e. -lr sign(g) wherever |g| >> eps; compare
        # where the oracle's gradient is clearly away from zero
        big = np.abs(og[name]) > 1e-3 * np.abs(og[name]).max()
        assert big.sum() > 100
        np.testing.assert_allclose(got[big], p_ref[big], rtol=0, atol=1e-6 * max(1.0, np.abs(p0).max()))


def test_sort_chunk_leaves_results_unchanged():
    g = synth.plain_scene(6000, seed=57)
    cams = _uneven_cameras()
    P = O.Params()
    a = ViewRun(g, cams, P)
    ws = B.Workspace(**capacity_for(g.n, cams))
    for chunk in (1024, 2048, 4096):
        ws.set_sort_chunk(chunk)
        b = ViewRun(g, cams, P, ws=ws)
        assert np.array_equal(a.sorted_vals, b.sorted_vals) and np.array_equal(a.ranges, b.ranges), chunk
        assert torch.equal(a.rgb, b.rgb) and np.array_equal(a.n_contrib, b.n_contrib), chunk
    with pytest.raises(B.GSError):
        ws.set_sort_chunk(1000)


def _mixed_cameras(n, seed, sizes=((64, 48), (128, 72), (192, 108), (256, 144), (384, 216))):
    rng = np.random.default_rng(seed)
    cams = []
    for k in range(n):
        w, h = sizes[rng.integers(len(sizes))]
        eye = (rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(-1.5, -0.2))
        cams.append(synth.look_at_camera(eye, (rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), 4.0),
                                         (0.0, -1.0, 0.0), w, h, rng.uniform(40.0, 80.0)))
    return cams


def test_each_view_of_a_batch_equals_its_render_alone():
    # 64 cameras of mixed resolution in one call; every view is bit-identical
    # to the same camera rendered on its own (per-tile lists keep the same
    # order: depth bits, then Gaussian index)
    g = synth.plain_scene(5000, seed=58)
    cams = _mixed_cameras(64, 59)
    P = O.Params()
    batch = ViewRun(g, cams, P)
    for k in (0, 7, 31, 63):
        alone = ViewRun(g, [cams[k]], P)
        assert np.array_equal(batch.image(k), alone.image(0)), k
        assert np.array_equal(batch.T_final(k), alone.T_final(0)), k


def test_autotuner_picks_and_caches(tmp_path):
    from paper_2605_13794_gb300.autotune import SORT_CHUNKS, TILE_SHAPES, Autotuner, max_tiles
    g = B.GaussianTensors.from_host(synth.plain_scene(6000, seed=60))
    cams = _mixed_cameras(8, 61)
    ws = B.Workspace(max_gaussians=g.n, max_records=g.n * len(cams), max_instances=64 * g.n * len(cams),
                     max_tiles=max_tiles(cams), max_pixels=sum(c.width * c.height for c in cams),
                     max_cameras=len(cams))
    path = str(tmp_path / "tune.json")
    choice = Autotuner(path).tune(ws, g, cams, B.RenderParams(), reps=2)
    assert (choice.tile_w, choice.tile_h) in TILE_SHAPES and choice.sort_chunk in SORT_CHUNKS
    assert len(choice.trials) == len(TILE_SHAPES) * len(SORT_CHUNKS)
    assert choice.ms == min(choice.trials.values())
    again = Autotuner(path).tune(ws, g, cams, B.RenderParams())  # from the cache file
    assert (again.tile_w, again.tile_h, again.sort_chunk) == (choice.tile_w, choice.tile_h, choice.sort_chunk)
    # the chosen configuration renders what the oracle renders with that tiling
    P = O.Params(tile_w=choice.tile_w, tile_h=choice.tile_h)
    run = ViewRun(synth.plain_scene(6000, seed=60), cams[:2], P)
    g64 = O.gaussians64(synth.plain_scene(6000, seed=60))
    for c in range(2):
        _compare_view(run, c, g64, cams[c], P)


def _small_request_camera(rng):
    w, h = [(64, 48), (128, 72), (192, 108), (256, 144)][rng.integers(4)]
    eye = (rng.uniform(-0.8, 0.8), rng.uniform(-0.8, 0.8), rng.uniform(-1.5, -0.2))
    return synth.look_at_camera(eye, (0.0, 0.0, 4.0), (0.0, -1.0, 0.0), w, h, 60.0)


def test_serving_batches_match_renders_alone():
    from paper_2605_13794_gb300.serve import Server, poisson_requests
    g_host = synth.plain_scene(5000, seed=62)
    g = B.GaussianTensors.from_host(g_host)
    reqs = poisson_requests(200.0, 1.0, _small_request_camera, seed=5)
    assert 150 < len(reqs) < 250
    server = Server(g, B.RenderParams(), key_budget_bytes=2e9, max_batch=16, max_pixels=16 * 256 * 144,
                    keep_images=True)
    stats = server.run(reqs, realtime=False)   # all waiting at once: full batches, three in flight
    assert stats["requests"] == len(reqs) and stats["batches"] >= len(reqs) // 16
    assert all(r.done is not None and r.latency >= 0 for r in reqs)
    assert 0 < stats["p50_ms"] <= stats["p99_ms"]
    # continuous batching: more than one batch on the device at once
    assert stats["slots"] == 3 and stats["max_in_flight"] >= 2 and stats["overlap_frac"] > 0
    P = O.Params()
    for r in (reqs[0], reqs[17], reqs[-1]):
        alone = ViewRun(g_host, [r.cam], P)
        assert torch.equal(r.image, alone.rgb), r.rid


def test_serving_splits_a_batch_that_overflows():
    from paper_2605_13794_gb300.serve import Server, poisson_requests
    g = B.GaussianTensors.from_host(synth.plain_scene(5000, seed=63))
    reqs = poisson_requests(200.0, 0.2, _small_request_camera, seed=6)
    # a key budget of 60k instances per slot with a low initial estimate:
    # batches overflow and are admitted again in smaller batches
    server = Server(g, B.RenderParams(), key_budget_bytes=3 * 24 * 60_000, max_batch=8, max_pixels=8 * 256 * 144,
                    inst_per_pixel=0.01, keep_images=True, slots=3)
    stats = server.run(reqs, realtime=False)
    assert stats["requests"] == len(reqs) and all(r.done is not None for r in reqs)
    assert stats["overflow_retries"] > 0
    P = O.Params()
    g_host = synth.plain_scene(5000, seed=63)
    for r in (reqs[0], reqs[-1]):
        assert torch.equal(r.image, ViewRun(g_host, [r.cam], P).rgb), r.rid
