"""The benchmark's JSON line and its roofline arithmetic, on the CPU.

The reference arm (the oracle on the host cores) runs a small workload end to
end and must print the one-line contract; the algorithmic-bytes helper must
give the per-update figures the roofline divides by.
"""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_per_gap_update():
    # 4 x 4 field, half the sites gaps, FP32: a sweep reads the other colour
    # once (8 sites x 4 B twice over the two half-steps = 64 B), reads and
    # writes the 8 gap sites (64 B) and reads the 16-bit mask (2 B): 130 B for
    # 8 updates.
    assert bench.bytes_per_gap_update(4.0, 0.5) == pytest.approx(130.0 / 8.0)
    assert bench.bytes_per_gap_update(4.0, 0.5) == pytest.approx(16.25)
    assert bench.bytes_per_gap_update(2.0, 0.5) == pytest.approx(8.25)
    # Every site a gap: each update reads its neighbours' colour once and
    # reads and writes itself, 3 s bytes, plus the mask.
    assert bench.bytes_per_gap_update(4.0, 1.0) == pytest.approx(12.125)


def test_calibration_iterations():
    class A:
        cal_iters = None
        cal_points = 2
    assert bench.cal_iters(A) == 16
    A.cal_points = 1
    assert bench.cal_iters(A) == 24
    A.cal_iters = 7
    assert bench.cal_iters(A) == 7
    # trisection's 16 iterations leave a narrower bracket than 24 bisections
    assert 3.0 ** -16 < 2.0 ** -24


def test_reference_arm_prints_the_contract_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "field128", "--steps", "2", "--warmup", "3"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "updates/s"
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert (d["n_gpus"], d["steps"], d["warmup"]) == (1, 2, 3)
    assert d["higher_is_better"] is True and d["scaling"] in ("weak", "strong")
    assert d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("field128")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"]
    assert cb["value"] == pytest.approx(d["value"])
    e2e = d["e2e"]
    assert e2e["value"] == pytest.approx(d["value"]) and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_batch_reference_arm_runs_our_config():
    """On a batch workload the reference arm (the oracle on the batch's
    smallest field) prints the config dict our own arm prints, so that the two
    lines describe one workload."""
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--workload", "slices32", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    args = bench.parse_args_for_tests(["--workload", "slices32"])
    assert d["config"] == bench.batch_config(args, 1)
    assert d["config"]["storage"] == "bf16" and d["config"]["fields"] == 32
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == pytest.approx(d["value"])
    assert "smallest" in d["cpu_baseline"]["sample"]
