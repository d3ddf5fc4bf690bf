"""bench.py's reference arm on the CPU: one JSON line with the requested step counts,
the GPU arm's config, metric and unit, and the oracle as its baseline."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert (d["steps"], d["warmup"]) == (1, 3)
    assert d["metric"] == bench.METRIC and d["unit"] == "input-samples/s" and d["higher_is_better"] is True
    assert d["config"] == bench.bench_config("BF_FP32_FFT")
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "input-samples/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_every_form_has_a_kernel_and_sources():
    for form in bench.FORM_NAMES.values():
        kernel = bench.FORM_KERNEL[form]
        for f in bench.KERNEL_SOURCES[kernel]:
            assert os.path.exists(os.path.join(ROOT, "paper_1702_04728_gb300", "csrc", f))
        assert len(bench.kernel_hash(kernel)) == 64
