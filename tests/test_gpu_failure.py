"""Failure detection on the GPU without a fault: a bounded device wait that
gives up returns, reports GS_ERR_TIMEOUT through the workspace's error word
(gs_sync_status), leaves every output inside its buffers and the context
usable, and the next call after gs_clear_error runs normally."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2605_13794_gb300 import binding as B
from paper_2605_13794_gb300 import synth
from tests.gpu_helpers import capacity_for, gpu_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2605_13794_gb300 import build
    build.build()
    assert torch.cuda.is_available()


def test_selection_sort_wait_gives_up_and_reports_timeout():
    g = synth.plain_scene(60000, seed=81)
    cam = synth.plain_camera(512, 512, 600.0)
    P = O.Params()
    ws = B.Workspace(**capacity_for(g.n, [cam]))
    gt = B.GaussianTensors.from_host(g)
    ws.preprocess(gt, [cam], gpu_params(P))
    ws.bin_sort()
    n, words = g.n, (g.n + 31) // 32
    assert ws.counts()["n_records"] > 20000  # a sort of many blocks
    ref = torch.zeros(words, dtype=torch.int32, device="cuda")
    ws.importance(cull_out=ref)
    ws.sync_status()
    # one poll per wait: a block that finds a predecessor not yet published gives up
    ws.set_spin_limit(1)
    timed_out = False
    for _ in range(20):
        cull = torch.zeros(words, dtype=torch.int32, device="cuda")
        ws.importance(cull_out=cull)
        c = ws.counts()  # reads the error word without raising
        if c["error"] == B.GS_ERR_TIMEOUT:
            timed_out = True
            break
        assert c["error"] == 0
    assert timed_out, "no look-back wait gave up in 20 tries"
    assert c["error_site"] == 3  # the radix sort's look-back
    with pytest.raises(B.GSError) as ei:
        ws.sync_status()
    assert ei.value.code == B.GS_ERR_TIMEOUT
    # the selection's later kernels skipped their work: every Gaussian stays culled
    assert synth.unpack_bits(cull.cpu().numpy().view(np.uint32), n).all()
    # cleared, with the default bound again, the next call runs normally
    ws.clear_error()
    ws.set_spin_limit(0)
    again = torch.zeros(words, dtype=torch.int32, device="cuda")
    ws.importance(cull_out=again)
    ws.sync_status()
    assert torch.equal(again, ref)
    ws.close()
