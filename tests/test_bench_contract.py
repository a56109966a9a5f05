"""bench.py's reference arm (the CPU oracle timed on the bench workload)
prints one JSON line with the keys the benchmark contract asks for; the
serving workload prints its 'unavailable' line.  CPU only."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    p = subprocess.run([sys.executable, "bench.py", *args], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run("--impl", "reference", "--workload", "c1", "--steps", "2", "--warmup", "3")
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    # the oracle needs no warm-up: the stream's first batches are timed (both
    # of the two asked for, each a few milliseconds on this graph)
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 0 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["higher_is_better"] is True and d["data"] == "synthetic"


def test_reference_arm_serving_is_unavailable():
    d = _run("--impl", "reference", "--workload", "c5")
    assert d["impl"] == "reference" and d["unavailable"]
