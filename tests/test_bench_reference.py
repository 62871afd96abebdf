"""The benchmark's reference arm on CPU (it times the FP64 oracle on the host
cores, no GPU): one JSON line with the contract's keys, the GPU arm's metric,
unit and config, one oracle sample per host core in each timed step, and the
extrapolation of the sample throughput to the full workload that the line
states."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_line():
    import bench
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == "ms/RHS" and line["higher_is_better"] is False
    assert line["config"] == bench.PROP_CONFIG
    assert line["steps"] == 1 and line["warmup"] == 1
    cpu = line["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "ms/RHS", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    # one sample per core in the timed step; the value is the sample throughput scaled to the
    # workload: wall / samples x preconditioner applications per RHS x volume ratio
    nsamp = cpu["cores"]
    assert cpu["sample"].startswith(f"{nsamp} samples")
    wall_s = line["ms_per_step"] * 1e-3 * line["steps"]
    assert abs(bench.oracle_extrapolation(wall_s, nsamp, bench.HEADLINE_CYCLES) - line["value"]) \
        <= 1e-9 * line["value"]
