"""bench.py's reference arm on CPU: the FP64 oracle timed on the host cores prints one JSON
line with the keys the benchmark contract asks for (metric, unit, value, steps, warm-up,
config, cpu_baseline of kind oracle, e2e with no host-device bytes), on a small lattice."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "64", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip().startswith("{")]
    assert len(lines) == 1, r.stdout
    out = json.loads(lines[0])
    import bench
    assert out["impl"] == "reference"
    assert out["metric"] == bench.METRIC and out["unit"] == "MLUPS"
    assert out["value"] > 0 and out["higher_is_better"] is True
    assert out["steps"] == 2 and out["warmup"] == 1 and out["n_gpus"] == 1
    assert out["dtype"] == "f64" and out["data"] == "synthetic"
    assert "workload" in out["config"]
    cb = out["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == out["value"] and cb["cores"] >= 1 and cb["sample"]
    assert cb["host"]["nproc"] >= cb["cores"] and cb["host"]["cpu_model"]
    e2e = out["e2e"]
    assert e2e["value"] == out["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert out["ms_per_step"] > 0
