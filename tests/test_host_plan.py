"""Host-side checks of the launch planner and workspace layout (no GPU): compiles
tests/host_plan_check.cu against libsfr.so and runs it.  The program checks, over many problem
sizes and SM counts, that the persistent tensor-core sweep's tile ranges and Delta V partial slots
are covered exactly once, that the SIMT splits and W-pass chunks cover the matrix, and that the
workspace buffers are aligned and do not overlap."""
import os
import shutil
import subprocess

import pytest

from paper_1503_03004_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_planner_and_workspace_invariants(tmp_path):
    nvcc = os.environ.get("NVCC", "nvcc")
    if shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    if not os.path.exists(binding.LIB_PATH):
        from paper_1503_03004_gb300 import build_lib
        build_lib.build()
    libdir = os.path.dirname(binding.LIB_PATH)
    exe = str(tmp_path / "host_plan_check")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-o", exe,
                        os.path.join(ROOT, "tests", "host_plan_check.cu"), "-L" + libdir, "-lsfr",
                        "-Xlinker", "-rpath=" + libdir], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-3000:]
