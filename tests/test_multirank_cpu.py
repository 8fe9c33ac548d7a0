"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas, no
data-path collective).  Each rank times the same work; the job's step time is
the slowest rank's and the job's rate counts every rank's units."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    ms = bench.max_over_ranks(10.0 + rank, w)      # rank r took 10 + r ms
    bench.barrier(w)
    rate = bench.job_rate(1000, ms, w)
    # the reference arm: only rank 0 does work, the others return at once
    skipped = bench.run_reference(None, w, r) is None if r != 0 else True
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"ms": ms, "rate": rate, "skipped": skipped}, f)
    import torch.distributed as dist
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms"] == 11.0                     # max over ranks, seen by every rank
        assert r["rate"] == pytest.approx(2 * 1000 / 11e-3)
        assert r["skipped"]


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.job_rate(2_073_600, 3.2, 1) == pytest.approx(2_073_600 / 3.2e-3)
