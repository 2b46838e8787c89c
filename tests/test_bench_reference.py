"""The benchmark's reference arm (the FP64 oracle on the host cores, its
uniform-grid search) runs without a GPU: its JSON line carries the
contract's keys, describes its own sample, and names the workload it
measured."""
import json
import os
import subprocess
import sys
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    with tempfile.TemporaryDirectory() as cache:
        out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                              "--workload", "halo", "--cpu-seconds", "1", "--cache-dir", cache], cwd=ROOT,
                             capture_output=True, text=True, timeout=600,
                             env={**os.environ, "CUDA_VISIBLE_DEVICES": ""})
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "rays/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 0
    assert line["config"]["workload"] == "halo_262144_nside1_l200kpc_F100"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle-grid" and cb["value"] == line["value"] and cb["cores"] >= 1 and "origins" in cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
