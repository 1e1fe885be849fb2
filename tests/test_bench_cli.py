"""The reference arm of bench.py (the FP64 oracle on the host cores) keeps the one-JSON-line
contract: impl, metric, value, unit, cpu_baseline and e2e for the workloads it times, an
`unavailable` line for the others.  CPU only; small cases."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


@pytest.mark.parametrize("workload", ["kpoints", "serving", "psweep"])
def test_reference_arm_unavailable_line(workload):
    d = _run("--workload", workload)
    assert d["impl"] == "reference" and d["unavailable"]


def test_reference_arm_fe_small_case():
    d = _run("--workload", "fe", "--fe-n", "4", "--steps", "1", "--warmup", "0")
    assert d["impl"] == "reference" and d["unit"] == "ms" and d["higher_is_better"] is False
    assert d["value"] > 0 and d["ms_per_step"] == d["value"]
    assert "4^3" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and "60 columns" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
