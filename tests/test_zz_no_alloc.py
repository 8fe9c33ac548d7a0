"""gs_visible_set_static: the Cull-column entry point that allocates nothing.

It serves callers that may not call cudaMalloc (a latency-critical serving
thread, a host callback, a plugin whose memory belongs to another allocator):
its scratch is a fixed device array of the library.  Its output must equal the
Cull column of the workspace path (gs_importance) for the same view, on two
calls in a row that share that scratch, and the 99 %-mass rule computed here
at the array's full size (2^20 Gaussians, with many equal and zero weights).
This file is collected last so that a run stopping at its first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _reference_view(B, ws, gt, cam, params, n):
    """w and the Cull column of one view through the workspace entry points."""
    ws.preprocess(gt, [cam], params)
    ws.bin_sort()
    w = torch.zeros(n, device="cuda")
    cull = torch.zeros((n + 31) // 32, dtype=torch.int32, device="cuda")
    ws.importance(w=w, cull_out=cull)
    ws.sync_status()
    return w, cull


def test_static_visible_set_matches_workspace_path():
    from paper_2605_13794_gb300 import binding as B
    from paper_2605_13794_gb300 import build, synth

    build.build()
    lib = B.lib()
    g = synth.plain_scene(20000, seed=61)
    gt = B.GaussianTensors.from_host(g)
    cams = [synth.plain_camera(256, 256, 300.0),
            synth.look_at_camera((0.4, -0.3, -0.6), (0.0, 0.0, 4.0), (0.0, -1.0, 0.0), 200, 160, 60.0)]
    ws = B.Workspace(max_gaussians=g.n, max_records=g.n, max_instances=64 * g.n, max_tiles=256, max_pixels=256 * 256)
    params = B.RenderParams()
    vis_mass = float(params.c().vis_mass)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for cam in cams:  # two calls in a row, the second reusing the scratch of the first
        w, cull_ref = _reference_view(B, ws, gt, cam, params, g.n)
        cull = torch.full_like(cull_ref, -1)  # stale contents: the call must overwrite every word
        cvis = torch.zeros(g.n, dtype=torch.int32, device="cuda")
        err = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        rc = lib.gs_visible_set_static(_p(w), g.n, vis_mass, _p(cull), _p(cvis), _p(err), stream)
        assert rc == B.GS_OK, lib.gs_last_error()
        torch.cuda.synchronize()
        assert err.item() == 0
        assert torch.equal(cull, cull_ref)
        visible = ~synth.unpack_bits(cull.cpu().numpy().view(np.uint32), g.n)
        assert np.array_equal(cvis.cpu().numpy() == 1, visible)
        assert 0 < visible.sum() < (w.cpu().numpy() > 0).sum() + 1
    # beyond the fixed scratch: rejected on the host with a clear error, nothing launched
    big = torch.zeros((1 << 20) + 1, device="cuda")
    rc = lib.gs_visible_set_static(_p(big), big.numel(), vis_mass, _p(cull), None, None, stream)
    assert rc == B.GS_ERR_CAPACITY
    assert b"at most 1048576" in lib.gs_last_error()


def test_static_visible_set_at_full_size_with_ties_and_zeros():
    """n = 2^20, the largest the fixed scratch takes: weights on a grid of
    2^-16 (exact in float, in the library's fixed-point sums and in FP64 sums
    here), a third of them zero and the rest drawn from 512 values, so that
    long runs of equal weights straddle the cut.  The column must equal the
    99 %-mass rule computed here: sort by w descending, ties toward the lower
    index, keep the prefix whose exclusive sum is below vis_mass of the total."""
    import oracle as O
    from paper_2605_13794_gb300 import binding as B
    from paper_2605_13794_gb300 import build, synth

    build.build()
    lib = B.lib()
    n = 1 << 20
    rng = np.random.default_rng(62)
    w_np = (rng.integers(1, 513, n) * 2.0 ** -16).astype(np.float32)
    w_np[rng.uniform(size=n) < 1 / 3] = 0.0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    w = torch.from_numpy(w_np).cuda()
    for vis_mass in (0.99, 0.5):  # two calls in a row on the shared scratch
        vm = float(np.float32(vis_mass))
        cull = torch.full(((n + 31) // 32,), -1, dtype=torch.int32, device="cuda")
        err = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        rc = lib.gs_visible_set_static(_p(w), n, vm, _p(cull), None, _p(err), stream)
        assert rc == B.GS_OK, lib.gs_last_error()
        torch.cuda.synchronize()
        assert err.item() == 0
        visible = ~synth.unpack_bits(cull.cpu().numpy().view(np.uint32), n)
        ref = O.visible_top_mass(w_np.astype(np.float64), vm)
        assert np.array_equal(visible, ref)
        assert not visible[w_np == 0].any()
