"""The reference arm of bench.py on CPU: `--impl reference` times the oracle
on a bounded sample of the bench workload and prints one JSON line with the
GPU arm's metric, unit and workload; under a multi-rank launch only rank 0
runs it."""
import json
import os
import subprocess
import sys
from pathlib import Path

import bench

ROOT = Path(__file__).resolve().parents[1]


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_line_of_the_bench_metric():
    lines = _run({"RANK": "0", "WORLD_SIZE": "1"})
    assert len(lines) == 1
    out = json.loads(lines[0])
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == bench.UNIT
    assert out["higher_is_better"] is True and out["steps"] == 1 and out["warmup"] == 1
    assert out["config"] == bench.bench_config(1)
    assert out["value"] > 0 and out["ms_per_step"] > 0
    # the line says what it measured: sampled time per step, and the full
    # iteration's rate extrapolated from it
    assert out["extrapolated"] is True
    ex = out["extrapolation"]
    assert ex["sampled_ms_per_step"] == out["ms_per_step"]
    assert abs(1e3 / ex["full_iteration_ms"] - out["value"]) <= 0.01 * out["value"]
    assert ex["full_iteration_ms"] > out["ms_per_step"] and ex["tiles_per_step"] == 64
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1
    assert cb["extrapolated"] is True
    assert cb["unit"] == bench.UNIT and cb["sample"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["unit"] == bench.UNIT
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_0_only():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []
