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


def test_flop_count_from_two_count_passes():
    """The rooflines count Σ over active points of (2m + k + 1), k the point's
    component order, from two count passes: A over the whole expansion and A1
    over its order <= 1 part, as (2m + 1) A + 2 (A - A1) + (A1 - n). That holds
    when the constant component contributes exactly one active point per query,
    in both forms; the per-order counts of the oracle (expansions cut at order
    0, 1 and 2) give the direct sum to compare with."""
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle as O
    import synth
    O.build()
    d, m = 4, 3
    c = synth.family_coeffs(synth.BASE_SEED + 71, m, d)
    fn = lambda dims, X: synth.family_cut(c, dims, X)
    X = synth.uniform_queries(synth.BASE_SEED + 71, 300, d)
    n = X.shape[0]
    for form in (0, 1):
        counts = []
        for order in (0, 1, 2):
            E = O.OracleDDSG(d, m)
            for u in O.full_order_components(d, order):
                E.add_regular(u, 3)
            E.fill_values(fn)
            E.hierarchize()
            counts.append(float(E.eval(X, form=form, want=("count",))["count"].astype(np.float64).sum()))
        assert counts[0] == n, (form, counts[0])            # one constant point per query
        A1, A = counts[1], counts[2]
        direct = (2 * m + 1) * counts[0] + (2 * m + 2) * (counts[1] - counts[0]) + (2 * m + 3) * (counts[2] - counts[1])
        assert (2.0 * m + 1.0) * A + 2.0 * (A - A1) + (A1 - n) == direct
