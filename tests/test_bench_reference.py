"""The benchmark's reference arm (the CPU oracle, no GPU needed): one JSON
line with the contract's keys, on the small Plummer workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "plummer", "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["workload"] == "plummer_n4096"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    # the step time is what ran (a sampled walk), the whole-pass scale is stated
    sc = d["scale"]
    assert sc["walk_scale"] >= 1 and sc["build_s"] > 0
    assert abs(sc["whole_pass_s"] - 4096 / d["value"]) <= 1e-9 * sc["whole_pass_s"]
    assert d["ms_per_step"] / 1e3 < sc["whole_pass_s"] * sc["walk_scale"]
    assert d["config"]["n_leaf"] == 16 and d["config"]["walk_group"] == 32


def test_bench_error_helpers_match_the_oracle_definitions():
    """The bench's own relative error and nearest-rank 99th percentile (used
    with the GPU direct sum) agree with the oracle's definitions."""
    import numpy as np

    import bench
    import oracle
    g = np.random.default_rng(3)
    for k in (1, 2, 99, 100, 101, 2048, 5000):
        a, ref = g.normal(size=(3, k)), g.normal(size=(3, k))
        e = bench._rel_err(a, ref)
        np.testing.assert_array_equal(e, oracle.rel_err(a, ref))
        assert bench._p99(e) == oracle.percentile(e, 0.99)
