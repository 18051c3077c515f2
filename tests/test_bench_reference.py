"""The benchmark's reference arms run on the CPU (the oracle) and print one
JSON line with the keys the bench contract asks for."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", *args],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    return json.loads(lines[0])


def _check(line, unit):
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == unit and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_reference_arm_descent():
    line = _run("--workload", "c1", "--steps", "2", "--warmup", "1", "--ref-seconds", "1.5")
    _check(line, "flip_evals/s")
    assert line["ms_per_step"] > 0 and line["cpu_baseline"]["nproc"] >= 1 and line["cpu_baseline"]["cpu_model"]


def test_reference_arm_headline_workload_is_bounded():
    """The default reference arm runs the headline workload (the 10^6-spin
    lattice) on a bounded sample and keeps to its time budget."""
    import time
    t0 = time.time()
    line = _run("--steps", "1", "--warmup", "0", "--ref-seconds", "2")
    _check(line, "flip_evals/s")
    assert line["config"]["workload"] == "c5"
    assert time.time() - t0 < 120


def test_reference_arm_pass_based_search():
    line = _run("--method", "fm", "--workload", "c1", "--steps", "2", "--warmup", "1", "--cpu-seconds", "1")
    _check(line, "moves/s")
    assert line["config"]["method"] == "fm" and line["ms_per_step"] > 0
