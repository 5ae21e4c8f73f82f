"""The reference arm of bench.py (the CPU oracle, timed) keeps the JSON
contract of the benchmark line: one line, the workload's metric and unit,
a cpu_baseline and an e2e object; workloads it does not time say so."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,sample", [("tess2000_100m", 20000), ("dist1024_100m", 4000),
                                             ("select256_500m", 20000)])
def test_reference_line(workload, sample):
    d = run("--workload", workload, "--steps", "2", "--warmup", "1", "--ref-sample", str(sample))
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "Gpoints/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["config"]["workload"] == workload and d["config"]["sample_points_per_step"] == sample
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


@pytest.mark.parametrize("workload", ["serve_1b", "count_4b"])
def test_reference_unavailable(workload):
    d = run("--workload", workload, "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and d["unavailable"]
