"""CPU checks of bench.py's contract: the reference arm (the float64 oracle on the host cores)
prints the JSON line the driver reads, and the committed ncu traffic summary still matches the
sweep kernel's source (bench.py reports roofline.traffic only while it does)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == "solves/s" and line["unit"] == "solves/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "solves/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "square16384_r64_bf16_mixed"


def test_committed_sweep_traffic_matches_the_kernel_source():
    t = bench.sweep_traffic(16384, 16384)
    assert t is not None, "profiles/sweep_tc_square8192_r64_bf16.md no longer matches the sweep kernel source"
    # DRAM traffic per launch is close to the 8 bytes per element the sweep must move
    assert 7.0 * 16384 ** 2 <= t <= 8.5 * 16384 ** 2
