"""The benchmark's reference arm on CPU: `bench.py --impl reference` times the
FP64 oracle on the bounded crop of the workload and prints one JSON line with
the same metric and unit as the GPU arm (no GPU involved)."""
import json
import os
import subprocess
import sys

from _util import ROOT


def _reference_line(*extra):
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3", *extra],
                         cwd=ROOT, capture_output=True, text=True, timeout=900,
                         env={**os.environ, "RANK": "0", "WORLD_SIZE": "1"})
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.strip().splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_prints_the_contract_line():
    line = _reference_line()
    assert line["impl"] == "reference"
    assert line["unit"] == "MLUPS" and line["higher_is_better"] is True and line["value"] > 0
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["metric"].startswith("fluid+thermal MLUPS")
    assert line["dtype"] == "f64" and line["data"] == "synthetic" and line["vs_baseline"] is None
    # the reference arm's end-to-end figure is its own value, with no device copies
    assert line["e2e"] == {"value": line["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and "sample" in cb
    assert "384^3" in line["config"]["workload"] and "crop" in line["config"]["sample"]


def test_reference_arm_other_ranks_print_nothing():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=300,
                         env={**os.environ, "RANK": "1", "WORLD_SIZE": "2"})
    assert out.returncode == 0, out.stderr[-2000:]
    assert not [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
