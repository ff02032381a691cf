"""bench.py's reference arm on the CPU: `--impl reference` times the FP64
oracle on the host cores and prints one JSON line with the keys the
benchmark contract fixes (metric, value, unit, steps, warm-up, timing,
scaling, dtype, data, config, cpu_baseline, e2e); the GPU arm is covered by
the GPU runs."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "unit", "ms_per_step", "scaling", "dtype", "data", "config"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 3 and d["n_gpus"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["dtype"] == "f64"
    assert d["data"] == "synthetic" and "core-shell" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the line's rate is the sample's histories over the timed steps
    per_step = int(d["config"]["workload"].split(" neutrons per step")[0].split(";")[-1].strip())
    assert abs(d["value"] - per_step / (d["ms_per_step"] * 1e-3)) <= 1e-9 * d["value"]
