"""The benchmark's reference arm (the FP64 oracle timed on the host cores)
runs without a GPU and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                          "--cpu-sample", "8"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    L = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in L, k
    assert L["impl"] == "reference" and L["value"] > 0 and L["unit"] == "shots/s"
    assert L["cpu_baseline"]["kind"] == "oracle" and L["cpu_baseline"]["cores"] >= 1
    assert L["e2e"]["h2d_bytes_per_step"] == 0 and L["e2e"]["d2h_bytes_per_step"] == 0
    assert L["config"]["workload"].startswith("ZSZ-LP-160")
