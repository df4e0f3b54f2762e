"""The reference arm of bench.py (the oracle timed on the host cores) prints the
benchmark contract's JSON line: one line, the metric, value and unit of the
workload, the step counts, a cpu_baseline describing the run and an e2e object
with no host-device traffic. Run here at tiny orders (host only, no GPU)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    env = dict(os.environ, WORLD_SIZE="1", RANK="0", LOCAL_RANK="0")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, env=env, cwd=ROOT, timeout=600, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload,n,dtype", [("single", 64, "f64+f32"), ("td", 32, "td+f64")])
def test_reference_line_keeps_the_contract(workload, n, dtype):
    d = _run("--workload", workload, "--steps", "2", "--warmup", "1", "--cpu-sample-n", str(n))
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["steps"] == 2 and d["warmup"] == 1 and d["n_gpus"] == 1
    assert d["unit"] == "s" and d["higher_is_better"] is False and d["value"] > 0
    assert abs(d["ms_per_step"] - 1e3 * d["value"]) <= 1e-6 * d["ms_per_step"]
    assert d["dtype"] == dtype and d["data"] == "synthetic"
    assert d["config"]["n"] == n and d["config"]["status"] == 0
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
