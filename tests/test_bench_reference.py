"""bench.py --impl reference on the CPU: the oracle timed on its bounded sample
prints the contract's JSON line (the same metric, unit and config as the GPU
arm, a cpu_baseline describing the run and an e2e entry with no copies)."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "s" and d["higher_is_better"] is False
    assert d["metric"].startswith("IFMM factor+solve") and d["steps"] == 1 and d["n_gpus"] == 1
    assert d["value"] > 0 and abs(d["ms_per_step"] - d["value"] * 1e3) < 1e-6 * d["ms_per_step"]
    assert d["config"]["workload"].startswith("bumpy131k")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and "sample" in cb and cb["value"] == d["value"]
    assert cb["sample_n"] * cb["scaled_by"] == 131072
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == "s"
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0
