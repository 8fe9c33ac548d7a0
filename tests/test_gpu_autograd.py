"""The differentiable render through torch.autograd: binding.render, whose
backward is the library's hand-written adjoint (gs_render_bwd behind a
torch.autograd.Function).  Its parameter gradients against the FP64 oracle's
(element-wise rule; row rule for the mean) and against central differences of
the oracle's forward on a tiny scene; a workspace that ran another forward
before the backward is refused."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_13794_gb300 import binding as B
from paper_2605_13794_gb300 import synth
from tests.gpu_helpers import (ViewRun, PARAM_NAMES, assert_gaussian_grads_close, assert_grad_close, capacity_for, gpu_params,
                               grads_to_host, oracle_view_matched)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_13794_gb300 import build
    build.build()
    O.build()
    assert torch.cuda.is_available()


def _leaf_gaussians(g):
    gt = B.GaussianTensors.from_host(g)
    for t in gt.params():
        t.requires_grad_(True)
    return gt


def _autograd_grads(g, cam, P, dL):
    """loss = sum(rgb * dL) through binding.render; returns the .grad tensors."""
    gt = _leaf_gaussians(g)
    ws = B.Workspace(**capacity_for(g.n, [cam]))
    rgb, T = B.render(ws, gt, [cam], gpu_params(P))
    assert rgb.requires_grad and not T.requires_grad
    loss = (rgb * torch.from_numpy(np.ascontiguousarray(dL, np.float32).ravel()).cuda()).sum()
    loss.backward()
    torch.cuda.synchronize()
    ws.sync_status()
    out = {k: t.grad.double().cpu().numpy() for k, t in zip(PARAM_NAMES, gt.params())}
    ws.close()
    return out, rgb.detach()


def test_autograd_gradients_match_the_oracle():
    g = synth.plain_scene(3000, seed=71)
    cam = synth.plain_camera(128, 112, 160.0)
    P = O.Params(bg=(0.1, 0.2, 0.3))
    dL = np.random.default_rng(72).standard_normal((3, cam.height, cam.width))
    gg, rgb = _autograd_grads(g, cam, P, dL)
    # the same gradients as a direct gs_render_bwd call on an equal forward
    run = ViewRun(g, [cam], P)
    direct = run.gt.zeros_like()
    run.ws.render_bwd(run.gt, torch.from_numpy(dL.astype(np.float32).ravel()).cuda(), direct, accumulate=False)
    run.ws.sync_status()
    dh = grads_to_host(direct)
    for k in PARAM_NAMES:
        assert np.array_equal(gg[k], dh[k]), k
    assert torch.equal(rgb, run.rgb)
    # and the oracle's
    g64 = O.gaussians64(g)
    fwd = oracle_view_matched(O, run, 0, g64, cam, P)
    og = O.grads_per_gaussian(O.backward_view(g64, fwd, cam, P, dL))
    assert_gaussian_grads_close(gg, og)


def _oracle_loss(g64, cam, P, dL):
    f = O.forward_view(g64, cam, P)
    st = (f["proj"]["status"].tobytes(), f["proj"]["rect"].tobytes(), f["n_contrib"].tobytes(),
          f["bins"][1].tobytes())
    return float((f["image"] * dL).sum()), st


@pytest.mark.parametrize("seed", [73, 74])
def test_autograd_gradients_match_central_differences(seed):
    """14 Gaussians in front of a 48 x 40 camera: every parameter's autograd
    gradient against the central difference (h = 1e-6 relative) of the FP64
    forward's loss, where no discrete decision moves within h (the gradient
    rule per tensor: 1e-3 of its largest entry, 1e-3 relative on entries above
    1 % of it)."""
    rng = np.random.default_rng(seed)
    g = synth.plain_scene(14, seed=seed)
    o = rng.uniform(0.05, 0.9, g.n)
    g.opacity_logit[:] = np.log(o / (1 - o)).astype(np.float32)
    g.mean[:, 0] = rng.uniform(-0.25, 0.25, g.n).astype(np.float32)
    g.mean[:, 1] = rng.uniform(-0.25, 0.25, g.n).astype(np.float32)
    g.mean[:, 2] = rng.uniform(2.0, 3.0, g.n).astype(np.float32)
    g.log_scale[:] = rng.uniform(np.log(0.01), np.log(0.04), (g.n, 3)).astype(np.float32)
    cam = synth.plain_camera(48, 40, 120.0)
    P = O.Params()
    dL = rng.standard_normal((3, cam.height, cam.width))
    gg, _ = _autograd_grads(g, cam, P, dL)
    g64 = O.gaussians64(g)
    L0, st0 = _oracle_loss(g64, cam, P, dL)
    layout = dict(mean=(g.n, 3), log_scale=(g.n, 3), quat=(g.n, 4), opacity_logit=(g.n,), sh=(g.n, 16, 3))
    checked = 0
    got_all, fd_all = {}, {}
    for name in PARAM_NAMES:
        arr = g64[name]                     # the oracle's attribute-major copy
        rows = arr.T if arr.ndim == 2 else (arr.transpose(2, 0, 1) if arr.ndim == 3 else arr)
        grad = gg[name].reshape(layout[name])
        idx = list(np.ndindex(*layout[name]))
        if name == "sh":
            idx = [idx[k] for k in rng.choice(len(idx), 120, replace=False)]
        for ix in idx:
            x0 = rows[ix]
            h = 1e-6 * max(1.0, abs(x0))
            rows[ix] = x0 + h
            Lp, stp = _oracle_loss(g64, cam, P, dL)
            rows[ix] = x0 - h
            Lm, stm = _oracle_loss(g64, cam, P, dL)
            rows[ix] = x0
            if stp != st0 or stm != st0:
                continue  # a discrete decision moved: no derivative there
            got_all.setdefault(name, []).append(grad[ix])
            fd_all.setdefault(name, []).append((Lp - Lm) / (2 * h))
            checked += 1
    assert checked > 0.9 * (g.n * 11 + 120)
    for name in PARAM_NAMES:
        assert_grad_close(name, np.array(got_all[name]), np.array(fd_all[name]))


def test_backward_after_another_forward_is_refused():
    g = synth.plain_scene(2000, seed=75)
    cam = synth.plain_camera(96, 80, 120.0)
    P = O.Params()
    ws = B.Workspace(**capacity_for(g.n, [cam]))
    a, b = _leaf_gaussians(g), _leaf_gaussians(g)
    rgb_a, _ = B.render(ws, a, [cam], gpu_params(P))
    rgb_b, _ = B.render(ws, b, [cam], gpu_params(P))
    with pytest.raises(RuntimeError, match="another forward"):
        rgb_a.sum().backward()
    rgb_b.sum().backward()   # the latest forward's backward is fine
    torch.cuda.synchronize()
    assert b.mean.grad is not None and torch.isfinite(b.mean.grad).all()
    ws.close()
