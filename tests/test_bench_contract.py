"""CPU checks of bench.py's contract: the reference arm (the float64 oracle on the host cores)
prints its one-line JSON result, and bench.py reports the committed ncu traffic figure of
the sweep kernel only while the kernel's source is the one the counters were taken from."""
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


def _summary():
    keys = ("traffic_bytes_per_element", "source", "source_until", "source_sha256", "helpers", "helpers_sha256")
    with open(os.path.join(ROOT, "profiles", "sweep_tc_square8192_r64_bf16.md")) as f:
        kv = dict(line.strip().split(": ", 1) for line in f if line.startswith("    ") and ": " in line
                  and line.strip().split(": ", 1)[0] in keys)
    assert set(kv) == set(keys), "the traffic summary lost one of its fields"
    return kv


def test_sweep_traffic_is_reported_only_for_the_captured_kernel_source():
    import hashlib
    kv = _summary()
    with open(os.path.join(ROOT, kv["source"]), encoding="utf-8") as f:
        text = f.read()
    region = text[:text.index(kv["source_until"])]
    with open(os.path.join(ROOT, kv["helpers"]), "rb") as f:
        helpers = f.read()
    same = (hashlib.sha256(region.encode("utf-8")).hexdigest() == kv["source_sha256"]
            and hashlib.sha256(helpers).hexdigest() == kv["helpers_sha256"])
    t = bench.sweep_traffic(16384, 16384)
    if same:
        # DRAM traffic per launch is close to the 8 bytes per element the sweep must move
        assert t is not None and 7.0 * 16384 ** 2 <= t <= 8.5 * 16384 ** 2
    else:
        # the kernel changed after the counters were taken: no traffic figure is reported
        assert t is None


def test_sweep_traffic_is_withheld_when_the_kernel_source_changes(tmp_path, monkeypatch):
    # a copy of the tree whose sweep source differs by one comment line
    kv = _summary()
    for rel in ("profiles/sweep_tc_square8192_r64_bf16.md", kv["source"], kv["helpers"]):
        dst = tmp_path / rel
        dst.parent.mkdir(parents=True, exist_ok=True)
        dst.write_bytes(open(os.path.join(ROOT, rel), "rb").read())
    src = tmp_path / kv["source"]
    src.write_text("// changed\n" + src.read_text(encoding="utf-8"), encoding="utf-8")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.sweep_traffic(16384, 16384) is None
