"""Parity at the benchmark's full size: 5M city Gaussians, one 1920x1080 aerial
view, LOD gate (d0 = 1600 m, Lmax = 5) and a Cull column, the launch
configuration bench.py times.  The FP64 oracle checks every active record and
tile list, the whole image, the parameter gradients of all Gaussians and the
importance outputs; projection decisions it flags as ties are checked to be
allowed outcomes and then taken from the GPU run."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_13794_gb300 import binding as B
from paper_2605_13794_gb300 import synth
from tests.gpu_helpers import (ViewRun, assert_grad_close, assert_gaussian_grads_close, assert_param_grad_close, assert_record_precision,
                               footprint_power_err, gpu_params, grads_to_host, oracle_view_matched, unpack_rect)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def city():
    from paper_2605_13794_gb300 import build
    build.build()
    O.build()
    g = synth.city_scene(5_000_000, seed=3)
    cam = synth.aerial_camera(seed=4)
    cull = synth.random_cull_bits(g.n, 0.2, seed=7)
    P = O.Params(lod_enable=True, lod_d0=1600.0, lod_Lmax=5, cull_enable=True)
    cap = dict(max_gaussians=g.n, max_records=400_000, max_instances=8_000_000, max_tiles=B.tiles_of(cam),
               max_pixels=cam.pixels, max_cameras=1)
    run = ViewRun(g, [cam], P, cull=cull, cap=cap)
    g64 = O.gaussians64(g)
    fwd = oracle_view_matched(O, run, 0, g64, cam, P, cull)
    return dict(g=g, cam=cam, cull=cull, P=P, run=run, g64=g64, fwd=fwd)


def test_fullsize_records_and_lists(city):
    run, fwd, g, cam = city["run"], city["fwd"], city["g"], city["cam"]
    pr = fwd["proj"]
    recs = run.records_of(0)
    both = np.nonzero(pr["status"] == O.ACTIVE)[0]
    assert sorted(recs.keys()) == both.tolist()
    assert len(both) > 50_000
    ridx = np.array([recs[i] for i in both], np.int64)
    assert np.array_equal(run.tt[ridx].astype(np.int64), pr["tiles"][both].astype(np.int64))
    assert_record_precision(run, ridx, pr, both, city["P"])
    perr = footprint_power_err(run.rd0[ridx], run.rd1[ridx], run.rd2[ridx], pr["conic"][both], pr["uv"][both])
    assert perr.max() <= 2e-4, perr.max()
    # every tile's sorted list, bit-exact: the oracle's binning of its decisions
    # and of the GPU's own FP32 records
    ts, lst = fwd["bins"]
    n = g.n
    own = dict(status=np.full(n, O.EMPTY, np.int8), rect=np.zeros((n, 4), np.int32),
               depth32=np.zeros(n, np.float32), tiles=np.zeros(n, np.int32))
    own["status"][both] = O.ACTIVE
    own["rect"][both] = unpack_rect(run.rect[ridx])
    own["depth32"][both] = run.depth_bits[ridx].view(np.float32)
    own["tiles"][both] = run.tt[ridx]
    ts2, lst2 = O.bin_tiles(own, cam, city["P"])
    for t, gl in enumerate(run.tile_lists(0)):
        assert np.array_equal(gl, lst[ts[t]:ts[t + 1]].astype(np.int64)), t
        assert np.array_equal(gl, lst2[ts2[t]:ts2[t + 1]].astype(np.int64)), t


def test_fullsize_image(city):
    run, fwd = city["run"], city["fwd"]
    # flagged pixels hold a fragment whose alpha or transmittance lies within
    # the FP32 error bound of a threshold: either decision there is correct
    ok = fwd["flags"] == 0
    assert ok.mean() > 0.999, ok.mean()
    err = np.abs(run.image(0) - fwd["image"]).max(axis=0)
    assert err[ok].max() <= 1e-4, err[ok].max()
    assert np.abs(run.T_final(0) - fwd["T"])[ok].max() <= 1e-4
    assert np.array_equal(run.n_contrib_img(0)[ok], fwd["n_contrib"][ok])


def test_fullsize_gradients(city):
    run, fwd, cam, g64 = city["run"], city["fwd"], city["cam"], city["g64"]
    rng = np.random.default_rng(9)
    dL = rng.standard_normal((3, cam.height, cam.width)) * 1e-3
    # a pixel's share of every gradient is linear in its dL/dC: with dL/dC = 0
    # at the flagged pixels, their undecided fragments add nothing on either side
    dL[:, fwd["flags"] != 0] = 0.0
    grads = run.gt.zeros_like()
    run.ws.render_bwd(run.gt, torch.from_numpy(dL.astype(np.float32).ravel()).cuda(), grads, accumulate=False)
    run.ws.sync_status()
    gg = grads_to_host(grads)
    og = O.grads_per_gaussian(O.backward_view(g64, fwd, cam, city["P"], dL))
    assert_gaussian_grads_close(gg, og)


def test_fullsize_importance(city):
    run, g, cam = city["run"], city["g"], city["cam"]
    # the scoring sweep: the training render's LOD gate, never the Cull column it recomputes
    P = O.Params(lod_enable=True, lod_d0=1600.0, lod_Lmax=5)
    run.ws.preprocess(run.gt, [cam], gpu_params(P))
    run.readback()
    n = g.n
    w = torch.zeros(n, device="cuda")
    a = torch.zeros(n, device="cuda", dtype=torch.int32)
    cull = torch.zeros((n + 31) // 32, device="cuda", dtype=torch.int32)
    run.ws.importance(w=w, a=a, cull_out=cull)
    run.ws.sync_status()
    fwd = oracle_view_matched(O, run, 0, city["g64"], cam, P)
    wg = w.double().cpu().numpy()
    ag = a.cpu().numpy().astype(np.int64)
    ao = fwd["a"].astype(np.int64)
    cnt = fwd["gcount"].astype(np.int64)
    free = cnt == 0
    assert free.sum() > 0.5 * (ao > 0).sum()
    # Gaussians on no flagged pixel: w within the gradient rule, a exact
    assert_grad_close("w", np.where(free, wg, 0.0), np.where(free, fwd["w"], 0.0))
    assert np.array_equal(ag[free], ao[free])
    # a flipped decision moves a by at most one and w by at most one
    # fragment's alpha * T (< 1e-2 at an alpha or T threshold) per flagged pixel
    assert np.all(np.abs(ag - ao) <= cnt)
    assert np.all(np.abs(wg - fwd["w"]) <= 1e-3 * np.abs(fwd["w"]) + 1e-2 * cnt + 1e-9)
    # the Cull column: the 99%-mass selection of the GPU's own w; the two
    # prefix sums (blocked on the GPU, sequential here) may round the cut one
    # place apart, never more
    vis = ~synth.unpack_bits(cull.cpu().numpy().view(np.uint32), n)
    w64 = w.cpu().numpy().astype(np.float64)
    mine = O.visible_top_mass(w64, float(np.float32(0.99)))
    pos = np.nonzero(w64 > 0)[0]
    order = pos[np.lexsort((pos, -w64[pos]))]
    k = int(mine.sum())
    diff = set(np.nonzero(vis != mine)[0].tolist())
    assert diff <= {int(order[k - 1]), int(order[min(k, len(order) - 1)])} and len(diff) <= 1, sorted(diff)[:10]
    assert fwd["w"][vis].sum() >= 0.99 * fwd["w"].sum() * (1 - 1e-3)
