"""bench.py's reference arm on the host: the FP64 oracle timed on a bounded
sample per step, printed as one JSON line with the benchmark's keys."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.timeout(300)
def test_reference_arm_prints_one_line_with_the_keys():
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1",
                        "--n", "100000"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [line for line in r.stdout.splitlines() if line.strip()]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["unit"] == "Mpix/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"] and d["config"]["gaussians"] == 100000
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


@pytest.mark.timeout(300)
def test_small_scene_oracle_on_one_thread_and_all_cores():
    """The small-scene oracle timing of the default line: a full step at one
    thread and as spawned processes on every host core."""
    sys.path.insert(0, ROOT)
    import bench
    r = bench.cpu_small_scene(steps=1)
    assert r["kind"] == "oracle" and r["unit"] == "Mpix/s"
    assert r["one_thread"]["cores"] == 1 and r["one_thread"]["value"] > 0
    assert r["all_cores"]["cores"] == (os.cpu_count() or 1) and r["all_cores"]["value"] > 0
