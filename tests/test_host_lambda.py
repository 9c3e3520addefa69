"""The smallest eigenvalue of B that sfr_solve reports (lambda_min_B, the SPD check of the
returned B) comes from a host routine (Householder tridiagonalisation and Sturm bisection).
This checks it against numpy's symmetric eigensolver on random, graded, near-degenerate,
indefinite and tiny matrices, compiling tests/host_lambda_check.cu against libsfr.so."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_1503_03004_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    rng = np.random.default_rng(5)
    out = []
    for r in (1, 2, 3, 5, 8, 25, 64):
        X = rng.standard_normal((r, r))
        out.append(X @ X.T + 1e-3 * np.eye(r))                     # SPD
        out.append(0.5 * (X + X.T))                                 # indefinite
        Q, _ = np.linalg.qr(rng.standard_normal((r, r)))
        lam = np.logspace(0, -10, r)                                # graded, condition 1e10
        out.append((Q * lam) @ Q.T)
        lam = 1.0 + 1e-9 * np.arange(r)                             # near-degenerate
        out.append((Q * lam) @ Q.T)
    out.append(np.diag([3.0, -2.0, 7.0, 0.5]))                      # diagonal
    out.append(np.zeros((4, 4)))
    return [0.5 * (A + A.T) for A in out]


def test_host_lambda_min_matches_eigvalsh(tmp_path):
    nvcc = os.environ.get("NVCC", "nvcc")
    if shutil.which(nvcc) is None:
        pytest.skip("nvcc not found")
    if not os.path.exists(binding.LIB_PATH):
        from paper_1503_03004_gb300 import build_lib
        build_lib.build()
    libdir = os.path.dirname(binding.LIB_PATH)
    exe = str(tmp_path / "host_lambda_check")
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-o", exe,
                        os.path.join(ROOT, "tests", "host_lambda_check.cu"), "-L" + libdir, "-lsfr",
                        "-Xlinker", "-rpath=" + libdir], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    cases = _cases()
    text = "".join(f"{A.shape[0]}\n" + " ".join(repr(float(x)) for x in A.ravel()) + "\n" for A in cases)
    r = subprocess.run([exe], input=text, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    got = [float(v) for v in r.stdout.split()]
    assert len(got) == len(cases)
    for A, g in zip(cases, got):
        w = np.linalg.eigvalsh(A)
        scale = max(1.0, float(np.abs(w).max())) if A.any() else 1.0
        assert abs(g - w[0]) <= 1e-12 * scale, (A.shape, g, w[0])
