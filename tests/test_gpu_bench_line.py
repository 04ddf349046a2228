"""bench.py end to end on the GPU: one short run of the default workload
prints one JSON line with every key of the measurement contract, a converged
solve and consistent units (a run of the whole script catches what the unit
tests of its helpers cannot, such as a variable of main() overwritten late)."""

import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_default_bench_line_has_the_contract_keys():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "3",
                          "--fp64-steps", "1"], capture_output=True, text=True, timeout=1200, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [x for x in out.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["unit"] == "s" and d["higher_is_better"] is False and d["n_gpus"] == 1
    assert abs(d["ms_per_step"] / 1e3 - d["value"]) < 1e-9 * max(1.0, d["value"])
    assert "workload" in d["config"] and d["gmres"]["relres"] <= 1e-8
    r = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in r, k
    assert abs(r["achieved"] / r["peak"] - r["frac"]) < 1e-9 and r["traffic"] and r["traffic"] > 0
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] > 0 and d["speedup_vs_fp64"] > 1.0
    assert d["error_vs_fp64"]["solution"] < 1e-7
