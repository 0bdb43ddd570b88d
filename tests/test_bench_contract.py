"""Host-side checks of bench.py (no GPU): the reference arm's JSON line
follows the bench contract, and the DRAM traffic figure of a kernel is
reported only while the kernel's source matches the committed capture."""
import hashlib
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"].startswith("MM iters/s")
    assert line["unit"] == "MM iters/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["n_gpus"] == 1
    assert line["steps"] == 1 and line["warmup"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("depth100k: P=100000 source, T=261104 target")
    # ms_per_step is time actually spent; the value is an estimate from the sample
    assert line["value_is_estimate"] is True and line["ms_per_step"] > 0
    assert line["estimated_seconds_per_pass"] > line["ms_per_step"] / 1e3


def test_traffic_is_null_once_the_kernel_source_changes(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    src = os.path.join(ROOT, "paper_2206_03410_gb300", "csrc", bench.KERNEL_SOURCES["solve_kernel"])
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    f = tmp_path / "traffic.txt"
    f.write_text("# comment\nsolve_kernel 12345 %s\nnn_kernel 777 0000000000000000\n" % digest)
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(f))
    assert bench.measured_traffic("solve_kernel") == 12345
    assert bench.measured_traffic("nn_kernel") is None        # source differs from the capture
    f.write_text("solve_kernel 12345 %s\n" % ("f" * 16))
    assert bench.measured_traffic("solve_kernel") is None
