"""gs_visible_set_static: the Cull-column entry point that allocates nothing.

It serves callers that may not call cudaMalloc (a latency-critical serving
thread, a host callback, a plugin whose memory belongs to another allocator):
its scratch is a fixed device array of the library.  Its output must equal the
Cull column of the workspace path (gs_importance) for the same view, on two
calls in a row that share that scratch.  This file is collected last so that a
run stopping at its first failure has already run every other test.
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
        rc = lib.gs_visible_set_static(_p(w), g.n, vis_mass, _p(cull), _p(cvis), stream)
        assert rc == B.GS_OK, lib.gs_last_error()
        torch.cuda.synchronize()
        assert torch.equal(cull, cull_ref)
        visible = ~synth.unpack_bits(cull.cpu().numpy().view(np.uint32), g.n)
        assert np.array_equal(cvis.cpu().numpy() == 1, visible)
        assert 0 < visible.sum() < (w.cpu().numpy() > 0).sum() + 1
    # beyond the fixed scratch: rejected on the host with a clear error, nothing launched
    big = torch.zeros((1 << 20) + 1, device="cuda")
    rc = lib.gs_visible_set_static(_p(big), big.numel(), vis_mass, _p(cull), None, stream)
    assert rc == B.GS_ERR_CAPACITY
    assert b"at most 1048576" in lib.gs_last_error()
