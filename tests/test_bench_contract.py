"""bench.py's host-side contracts, checked without a GPU: the reference arm
(the FP64 oracle timed on the host cores) prints one JSON line on rank 0 and
nothing on the other ranks, and the step's algorithmic-byte floor adds up to
the per-unit figures the bench line reports."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REF_ARGS = [sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0", "--cpu-rows", "4"]


def _run(env_extra=None):
    env = dict(os.environ)
    env.update(env_extra or {})
    return subprocess.run(REF_ARGS, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)


def test_reference_arm_prints_one_json_line():
    out = _run()
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["higher_is_better"] is True
    assert d["steps"] == 1 and d["warmup"] == 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == bench.WORKLOAD
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_print_nothing():
    out = _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]


def test_step_floor_bytes_per_unit():
    # one unit of each count at a time: 168 B per Gaussian, 240 per visible
    # pair, 192 per tile instance, 56 per pixel
    assert bench.step_floor_bytes(1, 0, 0, 0) == 168
    assert bench.step_floor_bytes(0, 1, 0, 0) == 240
    assert bench.step_floor_bytes(0, 0, 1, 0) == 192
    assert bench.step_floor_bytes(0, 0, 0, 1) == 56
    n, nv, m, p = 1_000_000, 170_306, 1_186_586, 816_000
    assert bench.step_floor_bytes(n, nv, m, p) == 168 * n + 240 * nv + 192 * m + 56 * p
