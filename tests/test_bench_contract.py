"""The bench's reference arm (the oracle on the host cores) keeps the JSON-line
contract: one line with the metric, value, unit, steps, timing fields, a
cpu_baseline describing the sample, an e2e object, and a sample no larger than
the workload. Runs on the CPU (the small d = 4 workload, one step)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _line(*args):
    r = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_reference_arm_line():
    d = _line("--impl", "reference", "--workload", "sg4", "--steps", "1", "--warmup", "0")
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "evals/s" and d["value"] > 0
    assert "d=4" in d["metric"] and d["steps"] == 1 and d["higher_is_better"] is True
    assert d["vs_baseline"] is None and d["dtype"] == "f64" and d["data"] == "synthetic"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert 1 <= d["config"]["queries_per_step"] <= 100_000     # never more than the workload


def test_headline_metric_is_verbatim_at_d100():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.metric_for(bench.WORKLOADS["d100"]) == \
        "interp evals/s (points·outputs) at d=100; % HBM roofline; FP32 vs FP64 error"
    assert "d=20" in bench.metric_for(bench.WORKLOADS["d20"])


def test_time_iteration_reference_arm_says_unavailable():
    d = _line("--impl", "reference", "--workload", "ti10", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and "unavailable" in d
