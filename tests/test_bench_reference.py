"""The reference arm of bench.py (the CPU oracle timed on the host cores):
one JSON line with the headline's metric and the fields the driver reads, on a
small grid so that it runs in seconds on the CPU."""

import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "24", "--steps", "2",
                        "--warmup", "1", "--ref-elements", "200"], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["config"]["elements"] == 2 * 24 * 24
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_whole_mesh_on_all_cores():
    """--ref-elements 0 (the default): every step is one whole right-hand side,
    timed on the oracle's threaded build with all host cores."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--n", "16", "--steps", "2",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    d = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][0])
    assert d["config"]["step"] == "one oracle right-hand side of all elements"
    assert d["cpu_baseline"]["cores"] == len(os.sched_getaffinity(0))
