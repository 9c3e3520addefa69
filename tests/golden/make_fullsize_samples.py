#!/usr/bin/env python3
"""Writes sampled outputs of the float64 oracle for the full-size workloads.

The oracle (oracle/fradm.py) cannot run inside the GPU tests at these sizes (minutes of CPU
time and tens of GB of host memory), so this script runs it once and stores, for a seeded
set of (i, j) positions, the oracle's L_ij and S_ij, plus its iteration count and ||L||_F.
It calls only `oracle/` and the seeded input generators; nothing here comes from the CUDA
path.  Usage (from the repository root):

    python tests/golden/make_fullsize_samples.py photometric   # 1048576 x 40, r = 3 (~2 min)
    python tests/golden/make_fullsize_samples.py square16384   # 16384 x 16384, r = 64 (~30 GB RAM)
    python tests/golden/make_fullsize_samples.py square16384_f32   # the same recipe stored in float32
    python tests/golden/make_fullsize_samples.py affinity   # 32768^2 FR-Nys, l = 2048 (~20 GB RAM)
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fradm as O  # noqa: E402
from paper_1503_03004_gb300 import synth  # noqa: E402

NSAMPLES = 4096

WORKLOADS = {
    # photometric-stereo stack: 1024 x 1024 pixels x 40 images, rank 3, float32 storage
    "photometric": dict(make=lambda: synth.photometric(side=1024, n_images=40, seed=1002), r=3,
                        kw=dict(rho=1.5, mu0=1.0, tol=1e-9, max_iter=300),
                        out="photometric_1048576x40_r3_samples.txt"),
    # the benchmark workload: 16384 x 16384, rank 64, 5% outliers in [-50, 50], bf16 storage
    "square16384": dict(make=lambda: synth.square_large(16384, 64, dtype="bf16", seed=1001), r=64,
                        kw=dict(rho=1.5, mu0=0.05, tol=1e-9, max_iter=300),
                        out="square16384_r64_bf16_samples.txt"),
    # the same recipe stored in float32: the workload of the float64 path at full size
    "square16384_f32": dict(make=lambda: synth.square_large(16384, 64, dtype="f32", seed=1001), r=64,
                            kw=dict(rho=1.5, mu0=0.05, tol=1e-9, max_iter=300),
                            out="square16384_r64_f32_samples.txt"),
    # spectral-clustering affinity, n = 32768, 20 clusters, bf16, through FR-Nys (Algorithm 2) with
    # l = 2048 sampled columns and the row shuffle synth.row_permutation(32768, 5)
    "affinity": dict(make=lambda: synth.affinity(n=32768, k=20, seed=1003, dtype="bf16"), r=20, nys_l=2048,
                     perm_seed=5, kw=dict(rho=1.5, mu0=1.0, tol=1e-9, max_iter=300),
                     out="affinity_32768_r20_nys2048_samples.txt"),
}


def sample_positions(m: int, n: int, seed: int = 4242):
    g = synth.rng(seed)
    return g.integers(0, m, NSAMPLES), g.integers(0, n, NSAMPLES)


def main(name: str) -> None:
    w = WORKLOADS[name]
    prob = w["make"]()
    M = prob.values_f64()
    m, n = M.shape
    ii, jj = sample_positions(m, n)
    t0 = time.time()
    if "nys_l" in w:
        perm = synth.row_permutation(m, w["perm_seed"])
        ref = O.fr_nys(M, w["r"], w["nys_l"], perm, sample=(ii, jj), **w["kw"])
        dt = time.time() - t0
        head = [f"# Float64 oracle (Algorithm 2, FR-Nys, l = {w['nys_l']}, row shuffle "
                f"synth.row_permutation({m}, {w['perm_seed']})) on {prob.name}, inner FR-ADM parameters {w['kw']}.",
                f"# oracle time {dt:.0f} s, blocks converged {bool(ref.left.converged)} / {bool(ref.top.converged)}.",
                f"iters {ref.left.iters + ref.top.iters}", f"iters_left {ref.left.iters}", f"iters_top {ref.top.iters}",
                "# columns: i j L_ij S_ij 0 (FR-Nys: S = M - L, no threshold)"]
        rows = zip(ii, jj, ref.L, ref.S, np.zeros(len(ii)))
    else:
        ref = O.fr_adm(M, w["r"], **w["kw"])
        dt = time.time() - t0
        z = M[ii, jj] - ref.L[ii, jj] + ref.Y_prev[ii, jj] / ref.mu_last
        head = [f"# Float64 oracle (Algorithm 1, FR-ADM) on {prob.name}, parameters {w['kw']}.",
                f"# oracle time {dt:.0f} s, converged {bool(ref.converged)}.",
                f"iters {ref.iters}", f"normL {np.linalg.norm(ref.L):.17g}", f"mu_last {ref.mu_last:.17g}",
                "# columns: i j L_ij S_ij z_ij (z = M - L + Y_prev / mu_last; S_ij is nonzero iff |z_ij| > 1/mu_last)"]
        rows = zip(ii, jj, ref.L[ii, jj], ref.S[ii, jj], z)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), w["out"])
    with open(path, "w") as f:
        f.write(head[0] + "\n")
        f.write("# Written by tests/golden/make_fullsize_samples.py (oracle and seeded inputs only);\n")
        for h in head[1:]:
            f.write(h + "\n")
        for a, b, lv, sv, zv in rows:
            f.write(f"{a} {b} {lv:.17g} {sv:.17g} {zv:.17g}\n")
    print(path, f"{dt:.0f} s")


if __name__ == "__main__":
    for arg in sys.argv[1:] or list(WORKLOADS):
        main(arg)
